// Internal layout of a UGKWP-LTS context on the device. Shared by the translation units of libugkwp.so.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include "../../include/ugkwp.h"

namespace ugk {

constexpr int kMaxIters = 256;   // face crossings + wall hits per particle per step
constexpr int kMaxNew = 2047;    // new particles per cell per step (11-bit index inside the particle id)
constexpr double kR = 0.5;       // gas constant in the reference units
constexpr double kRhoFloor = 1e-12;   // vacuum floor of the cell density (units of rho_inf)
constexpr int kTransportWarp = 1, kTransportStaged = 2;   // transport kernels (launch parameter)

// device error word bits
enum : int { ERR_LIMIT = 1, ERR_NONPHYS = 2, ERR_OVERFLOW = 4, ERR_CAPACITY = 8 };

// Per-cell face table used by the particle kernels: outward normal, plane offset (n.x <= d inside),
// dt_neighbour / dt_cell, and a packed word: face id (bits 0-23), local index of the face in the
// neighbour (24-25), boundary tag (26-28), 1 if the cell is the face's L side (bit 29). nbr < 0 on a
// boundary face.
template <typename T> struct alignas(16) CellFaces {
    T nx[4], ny[4], d[4], ratio[4];
    int nbr[4], meta[4];
};

template <typename T> struct ParticleSoA {
    T *x, *y, *u, *v, *w, *m;
    int32_t* cell;
    uint64_t* pid;
};

// fixed-size description of the per-step kernels' inputs (passed by value)
struct StepConsts {
    int C, F, dim, nwall, n_ref, wave_only, prec;
    int fx0, fx1, fx4;              // fixed-point exponents: mass, momentum, energy
    int fx_s2, fx_s3, shakhov;      // second / third velocity moments; Shakhov sampling (Pr != 1, particles)
    int n_f64, sort_every;          // faces in f64list; counting sort of the particles every sort_every steps
    int n_mix;                      // faces in mixlist
    int chunk;                      // particles per dynamically claimed chunk of the transport kernel
    int n_inj;                      // ghost particle sources (far-field and fixed faces)
    int order;                      // 2: second-order reconstruction for the wave fluxes
    int stag0, stag1;               // wall faces of the stagnation point (-1: none), for the monitors
    double mu_inf, omega, Pr, Tw, U_inf, m2RTw, sig_w;
    double wall_specular;           // Maxwell wall: specular fraction 1 - alpha (0: fully diffuse)
    double emx_cutoff;              // cells with e^{-x} below it sample no new particles (0: off)
    double T_cap, U_cap, T_min;     // realizability bounds of a cell state
    double W_inf[4], W_fix[4];
    uint32_t k0, k1;                // Philox key
};

// all device pointers of a context (trivially copyable: passed to kernels by value)
struct Dev {
    // geometry
    double *vol, *xc, *yc, *dt;
    double* rcp;                       // [2C] 1 / Omega_i, 1 / dt_i
    int* wallcell;                     // [C] 1: the cell has a wall face
    double *fax, *fay, *fex, *fey;     // [F] face start vertex a and edge b - a (1-D: the face point)
    int *inj_face, *inj_k;             // [n_inj] far-field / fixed faces (ghost particle sources), local index in L
    int* inj_n;                        // [n_inj] particles sampled by each source this step
    double* inj_par;                   // [5 n_inj] mass, ghost U, V, sqrt(R T), slab depth
    int* nfc;
    CellFaces<float>* cf32;
    CellFaces<double>* cf64;
    double* cshift;                    // [4C] periodic shift (1-D)
    double *cvx, *cvy;                 // [4C] vertices
    int *fL, *fR, *fbc, *fwall, *wall_face;
    double *fnx, *fny, *fs, *fdL, *fdR;
    int* face_f64;                     // 1: evaluate this face's flux in FP64 (production mode)
    // state
    double* W;                         // [4C]
    long long *wrt, *wprev, *wm, *wpl; // [5C]
    long long* wcol;                   // [5C] this step's collided particles that stay (retained = W^{p,+} - wcol)
    unsigned int* cross;               // [2F]
    long long* wallt;                  // [3 nwall]
    long long* frec;                   // [4F] record mode only (else null): crossing masses of the step, per face
                                       // and direction (L -> R, R -> L), before and after the scaling
    // per-step cell data
    double *tau, *xr, *emx, *Wh, *co, *mnew;
    double* samp;                      // [3C] U_i, V_i, R T_i of the new particles' distribution
    // production-mode wave fluxes: FP32 copies per cell, written once per step by k_flux_prep (second stream)
    float4 *w32, *wh32;                // W, W^h
    float4* dp32;                      // primitive perturbation (d rho, dU, dV, d theta) carrying W^h's remainder
    float* co32;                       // [8C] the 7 normalised coefficients (padded)
    double* grad;                      // [16C] order 2: limited gradients (d/dx, d/dy) of W's 4 components, then W^h's
    long long* whq;                    // [9C] Pr != 1: raw moments of the retained particles
    double* hq;                        // [3C] Pr != 1: acceptance-rejection weights a_x, a_y, M
    float* hq32;
    int *nhp, *nhp_off, *cnt, *off, *cur;
    int *scells, *nscell;              // cells with N^hp > 0 this step (in any order) and their number
    int *xq_i, *nxq;                   // production transport: slots queued by the stay pass for the flight pass
                                       // (bit 31: colliding) and their number
    float* xq_t;                       // their remaining free-flight times
    ParticleSoA<float> xq;             // their records as the stay pass read them (x, y, u, v, cell, id; w and m
                                       // unused), so that the flight pass reads them contiguously
    int* scan_tmp;
    double* flux;                      // [4F]
    double *res_part, *res;            // residual: per-block partials; [8] = raw of this step (4 used)
    double* chi_ema;
    double *surf_sum, *surf_last;      // [3 nwall]
    double* mon;                       // [8] monitored loads of the last step (C_d, C_H, stagnation C_p, C_Q) and
                                       // their EMAs
    // particles: A holds the cell-sorted retained set between steps, B is the staging buffer
    ParticleSoA<float> pa32, pb32;
    ParticleSoA<double> pa64, pb64;
    float *tau32, *dt32, *mnew32, *samp32;   // particle-precision copies of tau, dt, m_new, (U_i, V_i, R T_i),
    float* emx32;                            // e^{-dt/tau}
    float4* cst32;                           // per cell: (dt, e^{-dt/tau}, tau, face count as int bits), the
                                             // stay test's cell data in one 16-byte load
    long long* dstep;                  // step counter (Philox counter word)
    int* bufsel;                       // which particle buffer (A: 0, B: 1) holds the current particles
    int* flags;                        // [0]: this step sorts the particles by cell
    int *nretry, *retry;               // faces whose FP32 flux failed this step (re-evaluated in FP64)
    int* f64list;                      // faces always evaluated in FP64
    int* mixlist;                      // production mode: the faces of wall cells (FP32 moments, FP64 time integrals)
    unsigned int* done;                // blocks of k_update finished (last-block reduction)
    int* counts;                       // [0] retained, [1] new this step, [2] kept after the step, [3] capacity,
                                       // [4] processed, [5] chunk counter, [6] entered from ghosts, [7] their sort slots
    unsigned long long* stats;         // [0..7] per step (see ugkwp_stats), [8] surface samples,
                                       // [9] cumulative particle-steps, [10] cumulative new particles,
                                       // [11] cells set to the vacuum floor in the last step
    int* err;
};

// A block of a step kernel: its index and the number of blocks it is one of. A standalone launch passes
// (blockIdx.x, gridDim.x); the batched persistent kernel runs a case's stage as the same blocks, one after
// another on whichever CTA takes the work item, so that every per-block result (the residual partials) is that
// of the standalone launch.
struct VB {
    int b, n;
};
#define UGKWP_VB_LAUNCH (::ugk::VB{(int)blockIdx.x, (int)gridDim.x})

struct Ctx {
    StepConsts k{};
    Dev d{};
    int ni = 0, nj = 0, periodic_j = 0, capacity = 0, res_blocks = 0, grid_particles = 0, sms = 148;
    int device = -1;                             // the device current at creation (owns every allocation)
    int transport = 1;                           // transport kernel: kTransportWarp or kTransportStaged
    cudaStream_t stream = nullptr;
    void* (*dev_alloc)(size_t, void*, void*) = nullptr;   // caller's device allocator (null: cudaMalloc)
    void (*dev_free)(void*, void*) = nullptr;
    void* alloc_user = nullptr;
    cudaStream_t stream2 = nullptr;              // wave fluxes, overlapped with the particle kernels
    cudaStream_t stream3 = nullptr;              // ghost particle sources, overlapped with both
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join3 = nullptr;
    int64_t step = 0;
    double Kn = 0.0, Ma = 0.0;                   // case conditions (warm-start features)
    double res_scale[4] = {1.0, 1.0, 1.0, 1.0}; // freestream scale of the residual per component
    int use_graph = 0;
    cudaGraphExec_t graph = nullptr;
    std::string msg;
    std::vector<void*> allocs;
    int profiling = 0;
    std::vector<cudaEvent_t> prof_events;   // 2 kStages per profiled step (start, end of each stage)
};

constexpr int kStages = 6;   // decompose+scan, sample, particles, wave flux, sort, update+surface+close

// launchers implemented in ugkwp_flux.cu
// the wave-flux unit (ugkwp_flux.cuh, included by the core unit): launch_wave_flux(k, d, sms, stream) and
// flux_set_tables(tab, stream) with tab [5][20] the Taylor weights of phi1, psi2, psi3, beta, chi

}  // namespace ugk

struct ugkwp_ctx {
    ugk::Ctx c;
};
