// UGKWP-LTS steady-iteration step on one GPU: set-up, cell, particle and bookkeeping kernels and the C ABI.
//
// Compiled with -fmad=false: every floating-point operation on the particle path and in the cell
// decomposition is an individually rounded IEEE operation, in the order written, so that integer outcomes
// (cell indices, new-particle counts, fixed-point tallies) are reproducible bit for bit.
//
// Per step, on the context stream (all sizes device-resident, so one step can be captured in a graph):
//   k_begin_step       zero the step's crossing, wall and counter tallies; sort-step flag
//   k_decompose   a1   per cell: tau, W^p from the retained tally, W^h, e^{-dt/tau}, N^hp, coefficients
//   scan(N^hp)         new-particle slots (and the capacity check)
//   k_sample      a2   warp per cell: new particles appended after the retained ones, their W^{p,-}
//   k_particles   a3-a7 per particle: t_f, transport with dt_R/dt_L scaling, W^{p,+}, retained tally, removal
//                      (survivors compacted into the other particle buffer)
//   k_wave_flux   a9   per face (ugkwp_flux.cu): FP32 interior faces, FP64 wall/boundary faces
//   scan + k_scatter   every sort_every-th step: counting sort of the survivors by cell
//   k_update      a10, a11  per cell: Eq. 53, residual, particle-mass-ratio EMA; per wall face: p, tau_w, q;
//                      the last block closes the step
#include <cuda_runtime.h>
#include <math_constants.h>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>
#include "ugkwp_internal.h"
#include "ugkwp_detmath.cuh"
#include "ugkwp_flux.cuh"

namespace ugk {
namespace {

constexpr int kScanBlock = 1024;

// 2^e (|e| < 1022) from its exponent bits: the fixed-point scales with no FP64 arithmetic (B300's FP64 pipe is
// narrow); equal to ldexp(1.0, e)
__host__ __device__ __forceinline__ double pow2(int e)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)(e + 1023) << 52);
#else
    return ldexp(1.0, e);
#endif
}
#ifndef UGKWP_CHUNK
#define UGKWP_CHUNK 256
#endif
#ifndef UGKWP_SORT_EVERY
#define UGKWP_SORT_EVERY 8   // steps between counting sorts of the particles by cell
#endif
#ifndef UGKWP_PARTICLES_MINB
#ifndef UGKWP_FLY_MINB
#define UGKWP_FLY_MINB 6         // resident 128-thread blocks per SM the flight pass is compiled and launched for
#endif
#define UGKWP_PARTICLES_MINB 4   // resident 256-thread blocks per SM the warp-chunked transport kernel is compiled for
#endif
constexpr int kMaxCells = 1 << 20;

// ------------------------------------------------------------------------------------------ scan
__device__ __forceinline__ int block_excl_scan(int v, int* total)
{
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const int before = wid > 0 ? warp_sums[wid - 1] : 0;
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_blocks(const int* in, int* out, int* tmp, int n, const int* active)
{
    if (active && !*active) return;
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    int tot;
    const int e = block_excl_scan(i < n ? in[i] : 0, &tot);
    if (i < n) out[i] = e;
    if (threadIdx.x == 0) tmp[blockIdx.x] = tot;
}

// exclusive scan of the block totals (one block); out[n] and *total receive the grand total. With `cap`,
// the total is the number of new particles of the step: if the retained ones (cap[0]) plus them exceed the
// capacity (cap[3]) the error is flagged and none are sampled (the wave keeps that mass), so every slot the
// later kernels touch holds a valid particle; cap[4] receives the particles processed this step.
__global__ void k_scan_tops(int* tmp, int nb, int* out, int n, int* total, int* cap, int* err, const int* active)
{
    if (active && !*active) return;
    int tot;
    const int v = threadIdx.x < nb ? tmp[threadIdx.x] : 0;
    const int e = block_excl_scan(v, &tot);
    if (threadIdx.x < nb) tmp[threadIdx.x] = e;
    if (threadIdx.x == 0) {
        out[n] = tot;
        if (cap) {
            if ((long long)cap[0] + tot > (long long)cap[3]) {
                atomicOr(err, ERR_CAPACITY);
                tot = 0;
            }
            cap[4] = cap[0] + tot;
        }
        if (total) *total = tot;
    }
}

__global__ void k_scan_add(int* out, const int* tmp, int n, const int* active)
{
    if (active && !*active) return;
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) out[i] += tmp[blockIdx.x];
}

// exclusive scan of n ints (n <= 2^20); `active` (nullable) skips it when *active == 0
void exclusive_scan(const int* in, int* out, int* tmp, int n, int* total, cudaStream_t s, int* cap = nullptr,
                    int* err = nullptr, const int* active = nullptr)
{
    const int nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_blocks<<<nb, kScanBlock, 0, s>>>(in, out, tmp, n, active);
    k_scan_tops<<<1, kScanBlock, 0, s>>>(tmp, nb, out, n, total, cap, err, active);
    k_scan_add<<<nb, kScanBlock, 0, s>>>(out, tmp, n, active);
}

// ------------------------------------------------------------------------------ set-up (a0)
struct MeshDev {
    int ni, nj, dim, periodic_j, periodic_i, F;
    const double *xv, *yv;
    const int *bc_imin, *bc_imax, *bc_jmin, *bc_jmax;
};

__device__ __forceinline__ int vid(const MeshDev& m, int i, int j)
{
    return i + (m.ni + 1) * ((m.periodic_j && j == m.nj) ? 0 : j);
}

// one face: cells on each side (L always a fluid cell; n from L to R, outward from L on a boundary),
// boundary tag, unit normal, length, plane offset n.x = d
__global__ void k_setup_faces(const MeshDev m, Dev d, double* fd)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= m.F) return;
    const int ni = m.ni, nj = m.nj;
    if (m.dim == 1) {
        const double* xs = m.xv;
        d.fnx[f] = 1.0; d.fny[f] = 0.0; d.fs[f] = 1.0;
        d.fax[f] = xs[f]; d.fay[f] = 0.0; d.fex[f] = 0.0; d.fey[f] = 0.0;
        if (f == 0 && m.periodic_i) { d.fL[f] = ni - 1; d.fR[f] = 0; d.fbc[f] = UGKWP_BC_PERIODIC; fd[f] = xs[0]; }
        else if (f == 0) { d.fL[f] = 0; d.fR[f] = -1; d.fbc[f] = m.bc_imin[0]; d.fnx[f] = -1.0; fd[f] = -xs[0]; }
        else if (f == ni) { d.fL[f] = ni - 1; d.fR[f] = -1; d.fbc[f] = m.bc_imax[0]; fd[f] = xs[ni]; }
        else { d.fL[f] = f - 1; d.fR[f] = f; d.fbc[f] = 0; fd[f] = xs[f]; }
        return;
    }
    const int nif = (ni + 1) * nj;
    double nx, ny, len;
    int a;
    if (f < nif) {
        const int i = f % (ni + 1), j = f / (ni + 1);
        a = vid(m, i, j);
        const int b = vid(m, i, j + 1);
        const double ex = m.xv[b] - m.xv[a], ey = m.yv[b] - m.yv[a];
        d.fax[f] = m.xv[a]; d.fay[f] = m.yv[a]; d.fex[f] = ex; d.fey[f] = ey;
        len = sqrt(ex * ex + ey * ey);
        nx = ey / len; ny = -ex / len;
        if (i == 0) { nx = -nx; ny = -ny; d.fL[f] = i + ni * j; d.fR[f] = -1; d.fbc[f] = m.bc_imin[j]; }
        else if (i == ni) { d.fL[f] = (i - 1) + ni * j; d.fR[f] = -1; d.fbc[f] = m.bc_imax[j]; }
        else { d.fL[f] = (i - 1) + ni * j; d.fR[f] = i + ni * j; d.fbc[f] = 0; }
    } else {
        const int g = f - nif, i = g % ni, j = g / ni;
        a = vid(m, i, j);
        const int b = vid(m, i + 1, j);
        const double ex = m.xv[b] - m.xv[a], ey = m.yv[b] - m.yv[a];
        d.fax[f] = m.xv[a]; d.fay[f] = m.yv[a]; d.fex[f] = ex; d.fey[f] = ey;
        len = sqrt(ex * ex + ey * ey);
        nx = -ey / len; ny = ex / len;
        if (m.periodic_j) { d.fL[f] = i + ni * ((j + nj - 1) % nj); d.fR[f] = i + ni * j; d.fbc[f] = 0; }
        else if (j == 0) { nx = -nx; ny = -ny; d.fL[f] = i; d.fR[f] = -1; d.fbc[f] = m.bc_jmin[i]; }
        else if (j == nj) { d.fL[f] = i + ni * (nj - 1); d.fR[f] = -1; d.fbc[f] = m.bc_jmax[i]; }
        else { d.fL[f] = i + ni * (j - 1); d.fR[f] = i + ni * j; d.fbc[f] = 0; }
    }
    d.fs[f] = len;
    d.fnx[f] = nx; d.fny[f] = ny;
    fd[f] = nx * m.xv[a] + ny * m.yv[a];
}

// one cell: area, centroid, vertices, local faces (-i, +i, -j, +j) with outward normals and planes
__global__ void k_setup_cells(const MeshDev m, Dev d, const double* fd, int* cface, int* csgn, int* cnbr, int* cnk,
                              int* cbc, double* cnx, double* cny, double* cd)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int ni = m.ni, nj = m.nj;
    if (c >= ni * nj) return;
    if (m.dim == 1) {
        const double* xs = m.xv;
        const int i = c;
        d.vol[c] = xs[i + 1] - xs[i];
        d.xc[c] = 0.5 * (xs[i] + xs[i + 1]);
        d.yc[c] = 0.0;
        d.cvx[4 * c] = xs[i]; d.cvx[4 * c + 1] = xs[i + 1];
        d.nfc[c] = 2;
        const int q0 = 4 * c, q1 = 4 * c + 1;
        cface[q0] = (i == 0 && m.periodic_i) ? 0 : i;
        cface[q1] = (i == ni - 1 && m.periodic_i) ? 0 : i + 1;
        cnx[q0] = -1.0; cny[q0] = 0.0; cd[q0] = -xs[i];
        cnx[q1] = 1.0; cny[q1] = 0.0; cd[q1] = xs[i + 1];
        d.cshift[q0] = 0.0; d.cshift[q1] = 0.0;
        if (i > 0) { cnbr[q0] = i - 1; cnk[q0] = 1; csgn[q0] = -1; cbc[q0] = 0; }
        else if (m.periodic_i) { cnbr[q0] = ni - 1; cnk[q0] = 1; csgn[q0] = -1; cbc[q0] = UGKWP_BC_PERIODIC; d.cshift[q0] = xs[ni] - xs[0]; }
        else { cnbr[q0] = -1; cnk[q0] = 0; csgn[q0] = 1; cbc[q0] = m.bc_imin[0]; }
        if (i < ni - 1) { cnbr[q1] = i + 1; cnk[q1] = 0; csgn[q1] = 1; cbc[q1] = 0; }
        else if (m.periodic_i) { cnbr[q1] = 0; cnk[q1] = 0; csgn[q1] = 1; cbc[q1] = UGKWP_BC_PERIODIC; d.cshift[q1] = xs[0] - xs[ni]; }
        else { cnbr[q1] = -1; cnk[q1] = 0; csgn[q1] = 1; cbc[q1] = m.bc_imax[0]; }
        for (int k = 2; k < 4; ++k) { cface[4 * c + k] = 0; cnbr[4 * c + k] = -1; cnx[4 * c + k] = 0; cny[4 * c + k] = 0; cd[4 * c + k] = 0; cnk[4 * c + k] = 0; csgn[4 * c + k] = 1; cbc[4 * c + k] = 0; d.cshift[4 * c + k] = 0; }
        return;
    }
    const int i = c % ni, j = c / ni;
    const int v[4] = {vid(m, i, j), vid(m, i + 1, j), vid(m, i + 1, j + 1), vid(m, i, j + 1)};
    double X[4], Y[4];
    for (int q = 0; q < 4; ++q) {
        X[q] = m.xv[v[q]]; Y[q] = m.yv[v[q]];
        d.cvx[4 * c + q] = X[q]; d.cvy[4 * c + q] = Y[q];
    }
    d.vol[c] = 0.5 * ((X[2] - X[0]) * (Y[3] - Y[1]) - (X[3] - X[1]) * (Y[2] - Y[0]));
    const double A1 = 0.5 * ((X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]));
    const double A2 = 0.5 * ((X[2] - X[0]) * (Y[3] - Y[0]) - (X[3] - X[0]) * (Y[2] - Y[0]));
    d.xc[c] = (A1 * (X[0] + X[1] + X[2]) + A2 * (X[0] + X[2] + X[3])) / (3.0 * (A1 + A2));
    d.yc[c] = (A1 * (Y[0] + Y[1] + Y[2]) + A2 * (Y[0] + Y[2] + Y[3])) / (3.0 * (A1 + A2));
    d.nfc[c] = 4;
    const int nif = (ni + 1) * nj;
    const int jp = (m.periodic_j && j + 1 == nj) ? 0 : j + 1;
    const int fq[4] = {i + (ni + 1) * j, (i + 1) + (ni + 1) * j, nif + i + ni * j, nif + i + ni * jp};
    for (int k = 0; k < 4; ++k) {
        const int f = fq[k], q = 4 * c + k;
        const bool isL = d.fL[f] == c;
        cface[q] = f;
        csgn[q] = isL ? 1 : -1;
        cnx[q] = isL ? d.fnx[f] : -d.fnx[f];
        cny[q] = isL ? d.fny[f] : -d.fny[f];
        cd[q] = isL ? fd[f] : -fd[f];
        d.cshift[q] = 0.0;
        if (d.fR[f] < 0) { cnbr[q] = -1; cnk[q] = 0; cbc[q] = d.fbc[f]; }
        else { cnbr[q] = isL ? d.fR[f] : d.fL[f]; cnk[q] = k ^ 1; cbc[q] = 0; }
    }
}

__global__ void k_setup_face_dist(const MeshDev m, Dev d, const double* fd)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= m.F) return;
    const int L = d.fL[f], R = d.fR[f];
    if (m.dim == 1) {
        const double* xs = m.xv;
        if (d.fbc[f] == UGKWP_BC_PERIODIC) { d.fdL[f] = xs[m.ni] - d.xc[m.ni - 1]; d.fdR[f] = d.xc[0] - xs[0]; }
        else if (R < 0) { d.fdL[f] = d.fdR[f] = (f == 0) ? d.xc[0] - xs[0] : xs[m.ni] - d.xc[m.ni - 1]; }
        else { d.fdL[f] = xs[f] - d.xc[L]; d.fdR[f] = d.xc[R] - xs[f]; }
        return;
    }
    d.fdL[f] = fd[f] - (d.fnx[f] * d.xc[L] + d.fny[f] * d.yc[L]);
    d.fdR[f] = R >= 0 ? (d.fnx[f] * d.xc[R] + d.fny[f] * d.yc[R]) - fd[f] : d.fdL[f];
}

// ------------------------------------------------------------------ unstructured meshes (triangles, quads)
// Face and cell connectivity come from the host (ugkwp_create_unstructured); the geometry is computed here.
// A triangle is the degenerate quadrilateral (v0, v1, v2, v2): the quadrilateral's area, centroid and
// position-sampling formulas then give the triangle's.
struct UMeshDev {
    int C, F;
    const double *xv, *yv;
    const int* cv;                      // [4C] vertices, the third repeated in the fourth slot of a triangle
    const int *fa, *fb, *fl, *fr, *ftag;   // [F] edge a -> b (L's direction), sides, boundary tag
};

__global__ void k_setup_faces_u(const UMeshDev m, Dev d, double* fd)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= m.F) return;
    const int a = m.fa[f], b = m.fb[f];
    const double ex = m.xv[b] - m.xv[a], ey = m.yv[b] - m.yv[a];
    const double len = sqrt(ex * ex + ey * ey);
    d.fax[f] = m.xv[a]; d.fay[f] = m.yv[a]; d.fex[f] = ex; d.fey[f] = ey;
    d.fs[f] = len;
    const double nx = ey / len, ny = -ex / len;
    d.fnx[f] = nx; d.fny[f] = ny;
    d.fL[f] = m.fl[f]; d.fR[f] = m.fr[f]; d.fbc[f] = m.fr[f] < 0 ? m.ftag[f] : 0;
    fd[f] = nx * m.xv[a] + ny * m.yv[a];
}

// cell geometry and the outward normals / planes of its local faces (the integer tables are already set)
__global__ void k_setup_cells_u(const UMeshDev m, Dev d, const double* fd, const int* cface, const int* csgn,
                                double* cnx, double* cny, double* cd)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.C) return;
    double X[4], Y[4];
    for (int q = 0; q < 4; ++q) {
        X[q] = m.xv[m.cv[4 * c + q]]; Y[q] = m.yv[m.cv[4 * c + q]];
        d.cvx[4 * c + q] = X[q]; d.cvy[4 * c + q] = Y[q];
        d.cshift[4 * c + q] = 0.0;
    }
    d.vol[c] = 0.5 * ((X[2] - X[0]) * (Y[3] - Y[1]) - (X[3] - X[1]) * (Y[2] - Y[0]));
    const double A1 = 0.5 * ((X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]));
    const double A2 = 0.5 * ((X[2] - X[0]) * (Y[3] - Y[0]) - (X[3] - X[0]) * (Y[2] - Y[0]));
    d.xc[c] = (A1 * (X[0] + X[1] + X[2]) + A2 * (X[0] + X[2] + X[3])) / (3.0 * (A1 + A2));
    d.yc[c] = (A1 * (Y[0] + Y[1] + Y[2]) + A2 * (Y[0] + Y[2] + Y[3])) / (3.0 * (A1 + A2));
    for (int k = 0; k < 4; ++k) {
        const int q = 4 * c + k;
        if (k >= d.nfc[c]) { cnx[q] = 0.0; cny[q] = 0.0; cd[q] = 0.0; continue; }
        const int f = cface[q];
        const bool isL = csgn[q] > 0;
        cnx[q] = isL ? d.fnx[f] : -d.fnx[f];
        cny[q] = isL ? d.fny[f] : -d.fny[f];
        cd[q] = isL ? fd[f] : -fd[f];
    }
}

// Eq. 33 on the freestream field: dt_i = N_CFL Omega_i / ((|U_inf| + 3 sqrt(R T_inf)) sum_j s_j)
__global__ void k_setup_dt(Dev d, int C, const int* cface, double cfl, double cs, double* dtmin_part)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 1e300;
    if (c < C) {
        double perim = 0.0;
        for (int k = 0; k < d.nfc[c]; ++k) perim += d.fs[cface[4 * c + k]];
        const double dt = (cfl * d.vol[c]) / (cs * perim);
        d.dt[c] = dt;
        v = dt;
    }
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __shared__ double sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = sm[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fmin(b, sm[w]);
        dtmin_part[blockIdx.x] = b;
    }
}

// Eq. 34: dt_G = min dt_i, given to every cell under GTS
__global__ void k_setup_gts(Dev d, int C, const double* dtmin_part, int nb)
{
    double g = dtmin_part[0];
    for (int b = 1; b < nb; ++b) g = fmin(g, dtmin_part[b]);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) d.dt[c] = g;
}

__global__ void k_setup_tables(Dev d, int C, const int* cface, const int* csgn, const int* cnbr, const int* cnk,
                               const int* cbc, const double* cnx, const double* cny, const double* cd, int prod)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    d.rcp[2 * c] = 1.0 / d.vol[c];
    d.rcp[2 * c + 1] = 1.0 / d.dt[c];
    CellFaces<float> a;
    CellFaces<double> b;
    for (int k = 0; k < 4; ++k) {
        const int q = 4 * c + k;
        const int nb = (k < d.nfc[c]) ? cnbr[q] : -1;
        const double r = nb >= 0 ? d.dt[nb] / d.dt[c] : 1.0;
        const int meta = (cface[q] & 0xffffff) | ((cnk[q] & 3) << 24) | ((cbc[q] & 7) << 26) | ((csgn[q] > 0 ? 1 : 0) << 29);
        b.nx[k] = cnx[q]; b.ny[k] = cny[q]; b.d[k] = cd[q]; b.ratio[k] = r; b.nbr[k] = nb; b.meta[k] = meta;
        a.nx[k] = (float)cnx[q]; a.ny[k] = (float)cny[q]; a.d[k] = (float)cd[q]; a.ratio[k] = (float)r;
        a.nbr[k] = nb; a.meta[k] = meta;
    }
    d.cf32[c] = a;
    d.cf64[c] = b;
    // faces of a wall cell apply their time integrals in FP64 in production mode
    d.wallcell[c] = 0;
    for (int k = 0; k < d.nfc[c]; ++k)
        if (cbc[4 * c + k] == UGKWP_BC_WALL) {
            d.wallcell[c] = 1;
            for (int q = 0; q < d.nfc[c]; ++q) d.face_f64[cface[4 * c + q]] = 1;
        }
    (void)prod;
}

__global__ void k_wall_flags(const Dev d, int F, int* flag)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < F) flag[f] = d.fbc[f] == UGKWP_BC_WALL ? 1 : 0;
}

__global__ void k_wall_index(Dev d, int F, const int* idx)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    if (d.fbc[f] == UGKWP_BC_WALL) { d.fwall[f] = idx[f]; d.wall_face[idx[f]] = f; }
    else d.fwall[f] = -1;
}

// Realizable cell state: density above the vacuum floor, temperature in [T_min, T_cap] and speed at most
// U_cap (bounds fixed at creation from the freestream stagnation temperature, T_w and the fixed ghost
// temperature). Outside it the state is noise of a cell with (nearly) no gas.
__device__ __forceinline__ bool realizable(const StepConsts& K, const double* W)
{
    if (!(W[0] > kRhoFloor)) return false;
    const double r = 1.0 / W[0];   // one reciprocal (B300's FP64 pipe is narrow), as the CPU definition
    const double U = W[1] * r, V = W[2] * r;
    const double q = U * U + V * V;
    const double e = W[3] * r - 0.5 * q;
    if (!(e > 0.0)) return false;
    const double T = (e * (2.0 / 3.0)) * (1.0 / kR);
    return T >= K.T_min && T <= K.T_cap && q <= K.U_cap * K.U_cap;
}

// ------------------------------------------------------------------ a1: decomposition (Sec. IV B)
// e^x in float for the production decomposition (its own name: an overload here would hide the double
// dexp of the deterministic-math header from the calls in this namespace): x = k ln2 + r with ln 2 split in two (k ln2_hi exact),
// |r| <= ln2 / 2, Taylor series of e^r to r^7 (Horner), scaled by 2^k from the exponent bits; 0 below -87
// (Cody & Waite, "Software Manual for the Elementary Functions", 1980)
__device__ __forceinline__ float dexp_f32(float x)
{
    if (x < -87.0f) return 0.0f;
    if (x > 88.0f) return __int_as_float(0x7f800000);
    const float kf = rintf(__fmul_rn(x, 0x1.715476p+0f));
    const int k = (int)kf;
    const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(kf, 0x1.62e4p-1f)), __fmul_rn(kf, 0x1.7f7d1cp-20f));
    float p = 0x1.a01a02p-13f;                        // 1/7!
    p = __fadd_rn(0x1.6c16c2p-10f, __fmul_rn(r, p));  // 1/6!
    p = __fadd_rn(0x1.111112p-7f, __fmul_rn(r, p));   // 1/5!
    p = __fadd_rn(0x1.555556p-5f, __fmul_rn(r, p));   // 1/4!
    p = __fadd_rn(0x1.555556p-3f, __fmul_rn(r, p));   // 1/3!
    p = __fadd_rn(0.5f, __fmul_rn(r, p));
    p = __fadd_rn(1.0f, __fmul_rn(r, p));
    p = __fadd_rn(1.0f, __fmul_rn(r, p));
    return __fmul_rn(p, __int_as_float((k + 127) << 23));
}

// tau (below) in float (production precision, cells without a wall face); T = RT / R = 2 RT
__device__ __forceinline__ float tau_of_f32(const StepConsts& K, const double* W)
{
    const float rho = (float)W[0], r = __fdiv_rn(1.0f, rho);
    const float U = __fmul_rn((float)W[1], r), V = __fmul_rn((float)W[2], r);
    const float RT = __fmul_rn(__fsub_rn(__fmul_rn((float)W[3], r),
                                         __fmul_rn(0.5f, __fadd_rn(__fmul_rn(U, U), __fmul_rn(V, V)))),
                               0x1.555556p-1f);   // 2/3
    const float T = __fmul_rn(2.0f, RT);
    const float mu = __fmul_rn((float)K.mu_inf, dexp_f32(__fmul_rn((float)K.omega, dlog(T))));
    return __fdiv_rn(mu, __fmul_rn(rho, RT));
}

__device__ __forceinline__ double tau_of(const StepConsts& K, const double* W)
{
    // primitive variables through r = 1 / rho
    const double rho = W[0], r = 1.0 / rho, U = W[1] * r, V = W[2] * r;
    const double RT = (W[3] * r - 0.5 * (U * U + V * V)) * (2.0 / 3.0);
    const double T = RT / kR;
    const double mu = K.mu_inf * dpow(T, K.omega);
    return mu / (rho * RT);
}

// Taylor weights of the six entire functions behind the normalised coefficients, k = 0..19:
// 1/(k+1)!, 1/(k+2)!, 1/(k+3)!, (k+1)/(k+2)!, (k+1)/(k+3)!, (k+1)(k+2)/(2 (k+3)!)
constexpr int kSeries = 20;
__constant__ double c_series[6][kSeries];

// Normalised time-integration coefficients (Eq. 16 divided by dt, Eq. 48), x = dt/tau:
//   dbar_a = x psi2, dbar_b = -dt x beta, dbar_c = dt x psi3, dbar_d = phi1, dbar_e = -dt chi,
//   dbar_d - e^-x = x chi, dbar_e + dt e^-x / 2 = -dt x kappa, with phi1 = (1-e^-x)/x,
//   psi2 = (e^-x - 1 + x)/x^2, psi3 = (x^2/2 - x + 1 - e^-x)/x^3, chi = (phi1 - e^-x)/x,
//   beta = (1 + e^-x - 2 phi1)/x^2, kappa = (chi - e^-x/2)/x; Taylor series (Horner) for x < 1.
__device__ void lts_coeffs(double dt, double tau, double e, double* out)
{
    const double x = dt / tau;
    double phi1, psi2, psi3, chi, beta, kappa;
    if (x < 1.0) {
        const double mx = -x;
        phi1 = psi2 = psi3 = chi = beta = kappa = 0.0;
#pragma unroll
        for (int k = kSeries - 1; k >= 0; --k) {
            phi1 = fma(mx, phi1, c_series[0][k]);
            psi2 = fma(mx, psi2, c_series[1][k]);
            psi3 = fma(mx, psi3, c_series[2][k]);
            chi = fma(mx, chi, c_series[3][k]);
            beta = fma(mx, beta, c_series[4][k]);
            kappa = fma(mx, kappa, c_series[5][k]);
        }
    } else {
        phi1 = (1.0 - e) / x;
        psi2 = (e - 1.0 + x) / (x * x);
        psi3 = (0.5 * x * x - x + 1.0 - e) / (x * x * x);
        chi = (phi1 - e) / x;
        beta = (1.0 + e - 2.0 * phi1) / (x * x);
        kappa = (chi - 0.5 * e) / x;
    }
    out[0] = x * psi2;
    out[1] = -dt * x * beta;
    out[2] = dt * x * psi3;
    out[3] = phi1;
    out[4] = -dt * chi;
    out[5] = x * chi;
    out[6] = -dt * x * kappa;
}

// Shakhov acceptance-rejection weights of cell c (Eqs. 4-5): the heat flux Q_i of the particles retained in
// the cell at the start of the step, about the cell velocity U_i, from their raw moments (whq). The new
// particles follow the cell's g^S (Eq. 4 at U_i, T_i, Q_i): proposals c = sqrt(RT_i) z from the Maxwellian
// are accepted with probability (1 + psi) / M, psi = (a . z)(|z|^2 - 5), a = (1 - Pr) Q_i / (5 rho_i
// (RT_i)^(3/2)), M = 1 + 6 * 31 |a| (|z| <= 6 enforced by rejection). W has no z-momentum, so Q_z = 0; in 1-D
// also Q_y = 0. FP64, in the order of the CPU definition.
__device__ void shakhov_weights(const StepConsts& K, const Dev& d, int c, double RTi)
{
    const long long* h = d.whq + 9 * c;
    const double s0 = pow2(-K.fx0), s1 = pow2(-K.fx1), s2 = pow2(-K.fx_s2);
    const double s3 = pow2(-K.fx_s3);
    const double Sm = (double)h[0] * s0, Su = (double)h[1] * s1, Sv = (double)h[2] * s1;
    const double Suu = (double)h[3] * s2, Suv = (double)h[4] * s2, Svv = (double)h[5] * s2, Sq = (double)h[6] * s2;
    const double Suq = (double)h[7] * s3, Svq = (double)h[8] * s3;
    const double* W = d.W + 4 * c;
    const double U = W[1] / W[0], V = K.dim == 1 ? 0.0 : W[2] / W[0];
    const double UU = U * U + V * V;
    const double Ud = U * Su + V * Sv;
    const double cx3 = ((((Suq - 2.0 * (U * Suu + V * Suv)) + UU * Su) - U * Sq) + 2.0 * U * Ud) - U * UU * Sm;
    const double cy3 = ((((Svq - 2.0 * (U * Suv + V * Svv)) + UU * Sv) - V * Sq) + 2.0 * V * Ud) - V * UU * Sm;
    const double Qx = cx3 / (2.0 * d.vol[c]);
    const double Qy = K.dim == 1 ? 0.0 : cy3 / (2.0 * d.vol[c]);
    const double den = 5.0 * W[0] * (RTi * sqrt(RTi));
    const double ax = ((1.0 - K.Pr) * Qx) / den, ay = ((1.0 - K.Pr) * Qy) / den;
    const double M = 1.0 + 186.0 * sqrt(ax * ax + ay * ay);
    d.hq[3 * c] = ax; d.hq[3 * c + 1] = ay; d.hq[3 * c + 2] = M;
    d.hq32[3 * c] = (float)ax; d.hq32[3 * c + 1] = (float)ay; d.hq32[3 * c + 2] = (float)M;
}

// The same coefficients in FP32 (12 Taylor terms for x < 1, below FP32 resolution), for cells whose faces
// evaluate their fluxes in FP32 in production mode; the faces of wall cells keep the FP64 time integrals
constexpr int kSeries32 = 12;
__constant__ float c_series32[6][kSeries32];
__device__ void lts_coeffs_f32(float dt, float x, float e, float* out)
{
    float phi1, psi2, psi3, chi, beta, kappa;
    if (x < 1.0f) {
        const float mx = -x;
        phi1 = psi2 = psi3 = chi = beta = kappa = 0.0f;
#pragma unroll
        for (int k = kSeries32 - 1; k >= 0; --k) {
            phi1 = fmaf(mx, phi1, c_series32[0][k]);
            psi2 = fmaf(mx, psi2, c_series32[1][k]);
            psi3 = fmaf(mx, psi3, c_series32[2][k]);
            chi = fmaf(mx, chi, c_series32[3][k]);
            beta = fmaf(mx, beta, c_series32[4][k]);
            kappa = fmaf(mx, kappa, c_series32[5][k]);
        }
    } else {
        phi1 = (1.0f - e) / x;
        psi2 = (e - 1.0f + x) / (x * x);
        psi3 = (0.5f * x * x - x + 1.0f - e) / (x * x * x);
        chi = (phi1 - e) / x;
        beta = (1.0f + e - 2.0f * phi1) / (x * x);
        kappa = (chi - 0.5f * e) / x;
    }
    out[0] = x * psi2;
    out[1] = -dt * x * beta;
    out[2] = dt * x * psi3;
    out[3] = phi1;
    out[4] = -dt * chi;
    out[5] = x * chi;
    out[6] = -dt * x * kappa;
}

__device__ __forceinline__ void decompose_body(const VB vb, const StepConsts& K, const Dev& d)
{
    const int c = vb.b * blockDim.x + threadIdx.x;
    const unsigned am = __ballot_sync(0xffffffffu, c < K.C);   // the warp's lanes with a cell
    if (c >= K.C) return;
    const double* W = d.W + 4 * c;
    long long* r = d.wrt + 5 * c;
    const double vol = d.vol[c];
    const double s0 = pow2(-K.fx0), s1 = pow2(-K.fx1), s4 = pow2(-K.fx4);
    // production precision: tau, x = dt / tau and e^{-x} in FP32, except in cells with a wall face (stretched,
    // where the wave-flux time integrals need FP64) and at order 2 (whose g^h slope weight needs FP64)
    const bool f32 = K.prec == 0 && !d.wallcell[c] && K.order != 2;
    const double dt = d.dt[c];
    const float dt32 = (float)dt;
    double tau, x, e;
    float t32 = 0.0f, x32 = 0.0f, e32 = 0.0f;
    if (f32) {
        t32 = tau_of_f32(K, W);
        x32 = __fdiv_rn(dt32, t32);
        e32 = dexp_f32(-x32);
        tau = t32;
        x = x32;
        e = e32;
    } else {
        tau = tau_of(K, W);
        x = dt / tau;
        e = dexp(-x);
    }
    double Wp[4], Wh[4];
    // the factor 1 / Omega_i of Eq. 30 applied to the tally sums
    const double rvol = d.rcp[2 * c];
    Wp[0] = ((double)r[0] * s0) * rvol;
    Wp[1] = ((double)r[1] * s1) * rvol;
    Wp[2] = K.dim == 1 ? 0.0 : ((double)r[2] * s1) * rvol;
    Wp[3] = ((double)r[4] * s4) * rvol;
    // W^{p,-} of the retained particles is exactly the retained tally of the previous step (same particles,
    // masses, velocities and cell); k_sample adds the new particles. W^{p,+} starts from the same value
    // (every particle unchanged) and k_particles adds the changes; the retained tally of this step is
    // W^{p,+} minus the collided particles that stay (wcol), formed in k_update.
    for (int k = 0; k < 5; ++k) {
        d.wprev[5 * c + k] = r[k]; d.wm[5 * c + k] = r[k]; d.wpl[5 * c + k] = r[k]; d.wcol[5 * c + k] = 0;
    }
    for (int k = 0; k < 4; ++k) { Wh[k] = W[k] - Wp[k]; d.Wh[4 * c + k] = Wh[k]; }
    // FP32 cells keep tau, x, e^{-x} and the coefficients in FP32 only (the FP64 copies would cost conversions
    // on B300's narrow FP64 pipe; the cell-data read-back rebuilds them from the FP32 values). Order 2 weights
    // the slope term of g^h with dbar_e + dt e^{-x} / 2, whose FP32 closed form loses too many digits to
    // cancellation: FP64 coefficients for every cell then
    if (f32) {
        lts_coeffs_f32(dt32, x32, e32, d.co32 + 8 * (size_t)c);
    } else {
        d.tau[c] = tau;
        d.xr[c] = x;
        d.emx[c] = e;
        lts_coeffs(dt, tau, e, d.co + 7 * c);
        if (d.co32)
            for (int k = 0; k < 7; ++k) d.co32[8 * (size_t)c + k] = (float)d.co[7 * c + k];
    }
    int n = 0;
    double m = 0.0, Ui = 0.0, Vi = 0.0, RTi = 0.0;
    // W^hp = W^h e^{-dt_i/tau_i}; for rho^hp > 0: N^hp = ceil(rho^hp / rho N_ref), m = rho^hp Omega / N^hp
    // (Eqs. 25-26). The new particles' velocities follow the local distribution of the cell (Sec. III B), at
    // the cell velocity U_i and temperature T_i of the total W; the rest of W^h travels with the wave. A cell
    // whose e^{-x} is below the particle cutoff samples nothing (its W^h all travels with the wave)
    const double rho_hp = Wh[0] * e;
    if (!K.wave_only && rho_hp > 0.0 && !(e < K.emx_cutoff)) {
        const double q = ceil((rho_hp / W[0]) * (double)K.n_ref);
        if (q > (double)kMaxNew) {
            atomicOr(d.err, ERR_LIMIT);
        } else {
            n = (int)q;
            m = (rho_hp * vol) / q;
            const double rw = 1.0 / W[0];
            Ui = W[1] * rw;
            Vi = K.dim == 1 ? 0.0 : W[2] * rw;
            RTi = (W[3] * rw - 0.5 * (Ui * Ui + Vi * Vi)) * (2.0 / 3.0);
        }
    }
    if (K.shakhov && n > 0) shakhov_weights(K, d, c, RTi);
    // the cells that sample: appended to the list of k_sample, one slot range per warp
    const unsigned sm = __ballot_sync(am, n > 0);
    if (sm) {
        const int leader = __ffs(am) - 1, lane = threadIdx.x & 31;
        int base = 0;
        if (lane == leader) base = atomicAdd(d.nscell, __popc(sm));
        base = __shfl_sync(am, base, leader);
        if (n > 0) d.scells[base + __popc(sm & ((1u << lane) - 1u))] = c;
    }
    d.nhp[c] = n;
    d.mnew[c] = m;
    d.samp[3 * c] = Ui; d.samp[3 * c + 1] = Vi; d.samp[3 * c + 2] = RTi;
    if (!f32) {
        t32 = (float)tau;
        e32 = (float)e;
    }
    d.tau32[c] = t32;
    d.emx32[c] = e32;
    d.dt32[c] = dt32;
    if (d.cst32) d.cst32[c] = make_float4(dt32, e32, t32, __int_as_float(d.nfc[c]));
    if (n > 0) {
        d.mnew32[c] = (float)m;
        d.samp32[3 * c] = (float)Ui; d.samp32[3 * c + 1] = (float)Vi; d.samp32[3 * c + 2] = (float)RTi;
    } else {
        d.mnew32[c] = 0.0f;
        d.samp32[3 * c] = 0.0f; d.samp32[3 * c + 1] = 0.0f; d.samp32[3 * c + 2] = 0.0f;
    }
    d.cnt[c] = 0;
    d.cur[c] = 0;
}
__global__ void k_decompose(const StepConsts K, Dev d) { decompose_body(UGKWP_VB_LAUNCH, K, d); }

// ------------------------------------------------- a8: second-order reconstruction (order 2)
// Limited gradients (d/dx, d/dy) of the four components of W (v = 0..3) and W^h (v = 4..7) of one cell (FP64).
// 1-D: a smooth (van Albada type) limiter of the one-sided slopes a, b to the two neighbours (zero next to a
// boundary face), ((b^2 + e2) a + (a^2 + e2) b) / (a^2 + b^2 + 2 e2), e2 = K^3 h s^2 (K, s as below, h the
// cell length): exact for a = b, zero for a = -b and differentiable, so that steady runs converge.
// 2-D: least-squares gradient over the neighbours across interior and periodic faces, weights 1 / |dx|^2
// (zero with fewer than two), then Venkatakrishnan's limiter (a smooth form of keeping the reconstruction at
// every face midpoint within the values of the cell and those neighbours), one factor per component, the
// smallest over the faces and at most 1, epsilon^2 = (K h)^3 s^2 with K = 5, h = sqrt(Omega) and s the
// component's freestream scale (rho_inf, rho_inf (U_inf + sqrt(R T_inf)), (rho E)_inf).
__device__ __forceinline__ double smooth_slope(double a, double b, double e2)
{
    return ((b * b + e2) * a + (a * a + e2) * b) / ((a * a + b * b) + 2.0 * e2);
}

// one thread per (cell, component): eight independent FP64 chains per cell keep the FP64 pipe busier than
// one thread walking them in turn
__global__ void k_gradients(const StepConsts K, Dev d)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * K.C) return;
    const int c = t >> 3;
    const CellFaces<double>& F = d.cf64[c];
    const int nf = d.nfc[c];
    double* g = d.grad + 16 * (size_t)c;
    {
        const int v = t & 7;
        const double* A = v < 4 ? d.W : d.Wh;
        const int comp = v & 3;
        const double vc = A[4 * c + comp];
        double gx = 0.0, gy = 0.0;
        if (K.dim == 1) {
            const int nl = F.nbr[0], nr = F.nbr[1];
            if (nl >= 0 && nr >= 0) {
                // a neighbour across a periodic face, in this cell's frame
                const double xl = d.xc[nl] - d.cshift[4 * c], xr = d.xc[nr] - d.cshift[4 * c + 1];
                const double sc = comp == 0 ? K.W_inf[0] : comp == 3 ? K.W_inf[3] : K.W_inf[0] * (K.U_inf + sqrt(kR));
                gx = smooth_slope((vc - A[4 * nl + comp]) / (d.xc[c] - xl), (A[4 * nr + comp] - vc) / (xr - d.xc[c]),
                                  (125.0 * d.vol[c]) * (sc * sc));
            }
        } else {
            double a11 = 0.0, a12 = 0.0, a22 = 0.0, b1 = 0.0, b2 = 0.0, vmax = vc, vmin = vc;
            int nn = 0;
            for (int k = 0; k < nf; ++k) {
                const int nb = F.nbr[k];
                if (nb < 0) continue;
                const double dx = d.xc[nb] - d.xc[c], dy = d.yc[nb] - d.yc[c];
                const double w = 1.0 / (dx * dx + dy * dy), dv = A[4 * nb + comp] - vc;
                a11 += w * dx * dx; a12 += w * dx * dy; a22 += w * dy * dy;
                b1 += w * dx * dv; b2 += w * dy * dv;
                if (A[4 * nb + comp] > vmax) vmax = A[4 * nb + comp];
                if (A[4 * nb + comp] < vmin) vmin = A[4 * nb + comp];
                nn++;
            }
            const double det = a11 * a22 - a12 * a12;
            if (nn >= 2 && det > 1e-12 * (a11 * a22)) {
                gx = (a22 * b1 - a12 * b2) / det;
                gy = (a11 * b2 - a12 * b1) / det;
                const double sc = comp == 0 ? K.W_inf[0] : comp == 3 ? K.W_inf[3] : K.W_inf[0] * (K.U_inf + sqrt(kR));
                const double kh = 5.0 * sqrt(d.vol[c]);
                const double eps2 = ((kh * kh) * kh) * (sc * sc);
                double phi = 1.0;
                for (int k = 0; k < nf; ++k) {
                    const int f = F.meta[k] & 0xffffff;
                    const double mx = d.fax[f] + 0.5 * d.fex[f], my = d.fay[f] + 0.5 * d.fey[f];
                    const double d2 = gx * (mx - d.xc[c]) + gy * (my - d.yc[c]);
                    if (d2 == 0.0) continue;
                    const double d1 = d2 > 0.0 ? vmax - vc : vmin - vc;
                    const double r = ((d1 * d1 + eps2) * d2 + (2.0 * d2) * (d2 * d1)) /
                                     (d2 * (((d1 * d1 + 2.0 * (d2 * d2)) + d1 * d2) + eps2));
                    if (r < phi) phi = r;
                }
                gx *= phi;
                gy *= phi;
            }
        }
        g[2 * v] = gx;
        g[2 * v + 1] = gy;
    }
}

// per-step zeroing of face crossings, wall tallies and counters; the sort flag of this step
__device__ __forceinline__ void begin_body(const VB vb, const StepConsts& K, const Dev& d)
{
    const int t = vb.b * blockDim.x + threadIdx.x, nt = vb.n * blockDim.x;
    for (int q = t; q < 2 * K.F; q += nt) d.cross[q] = 0u;
    for (int q = t; q < 3 * K.nwall; q += nt) d.wallt[q] = 0;
    if (d.frec)
        for (int q = t; q < 4 * K.F; q += nt) d.frec[q] = 0;
    if (K.shakhov)
        for (int q = t; q < 9 * K.C; q += nt) d.whq[q] = 0;
    if (t == 0) {
        for (int k = 2; k < 8; ++k) d.stats[k] = 0;
        d.stats[11] = 0;
        d.stats[12] = 0;
        d.counts[2] = 0;
        d.counts[5] = 0;
        d.counts[6] = 0;
        d.counts[7] = 0;
        d.stats[13] = 0;
        *d.nretry = 0;
        *d.nscell = 0;
        if (d.nxq) *d.nxq = 0;
        *d.done = 0u;
        // a counting sort every sort_every-th step, whenever holes (removed particles, updated in place) fill
        // more than a quarter of the slots, and whenever the slots fill more than seven eighths of the capacity
        // (so that holes do not use up room the new particles need)
        const long long slots = d.counts[0], alive = (long long)d.stats[1], cap = d.counts[3];
        d.flags[0] = (int)(*d.dstep % K.sort_every == (long long)(K.sort_every - 1) || 4 * (slots - alive) > slots ||
                           8 * slots > 7 * cap);
    }
}
__global__ void k_begin_step(const StepConsts K, Dev d) { begin_body(UGKWP_VB_LAUNCH, K, d); }

// per-cell particle-precision views
template <typename T> struct PCell;
template <> struct PCell<float> {
    const float *tau, *dt, *mnew, *samp, *hq, *emx;
    __device__ float tau_(int c) const { return tau[c]; }
    __device__ float emx_(int c) const { return emx[c]; }
    __device__ float q_(int c, int k) const { return hq[3 * c + k]; }
    __device__ float dt_(int c) const { return dt[c]; }
    __device__ float m_(int c) const { return mnew[c]; }
    __device__ float s_(int c, int k) const { return samp[3 * c + k]; }
};
template <> struct PCell<double> {
    const double *tau, *dt, *mnew, *samp, *hq, *emx;
    __device__ double tau_(int c) const { return tau[c]; }
    __device__ double emx_(int c) const { return emx[c]; }
    __device__ double q_(int c, int k) const { return hq[3 * c + k]; }
    __device__ double dt_(int c) const { return dt[c]; }
    __device__ double m_(int c) const { return mnew[c]; }
    __device__ double s_(int c, int k) const { return samp[3 * c + k]; }
};

__device__ __forceinline__ float fsqrt_(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ double fsqrt_(double x) { return __dsqrt_rn(x); }
// float -> int64, IEEE round-half-even, with 32-bit integer operations only (B300 executes 64-bit
// float<->integer conversions on its narrow FP64 pipe). Exact for |x| < 2^63.
__device__ __forceinline__ long long rint_ll(float x)
{
    const uint32_t b = __float_as_uint(x);
    const int ex = (int)((b >> 23) & 0xffu);
    if (ex == 0) return 0;
    const uint32_t mant = (b & 0x7fffffu) | 0x800000u;
    const int sh = ex - 150;                 // |x| = mant 2^sh
    long long r;
    if (sh >= 0) {
        r = (long long)mant << sh;
    } else if (sh >= -24) {
        const int k = -sh;
        uint32_t q = mant >> k;
        const uint32_t rem = mant & ((1u << k) - 1u), half = 1u << (k - 1);
        if (rem > half || (rem == half && (q & 1u))) q += 1u;
        r = (long long)q;
    } else {
        r = 0;
    }
    return (b >> 31) ? -r : r;
}
__device__ __forceinline__ long long rint_ll(double x) { return __double2ll_rn(x); }

// ----------------------------------------------------------- fixed-point tallies (Eq. 30)
template <typename T>
__device__ __forceinline__ long long fixp(T v, T scale, int* err)
{
    const T s = v * scale;
    if (!(fabs(s) < T(4.611686018427387904e18))) { atomicOr(err, ERR_OVERFLOW); return 0; }
    return rint_ll(s);
}

// the five tallied moments of one particle, m (1, u, v, w, |u|^2/2), as fixed-point integers
template <typename T>
__device__ __forceinline__ void fix5(T m, T u, T v, T w, T s0, T s1, T s4, int* err, long long o[5])
{
    const T e = T(0.5) * ((u * u + v * v) + w * w);
    o[0] = fixp(m, s0, err);
    o[1] = fixp(m * u, s1, err);
    o[2] = fixp(m * v, s1, err);
    o[3] = fixp(m * w, s1, err);
    o[4] = fixp(m * e, s4, err);
}

// Pr != 1: raw velocity moments m (1, u, v, uu, uv, vv, q, uq, vq), q = |u|^2, of the particles retained at
// the start of the step, per cell, as fixed-point integers (the Shakhov heat flux of the sampling)
template <typename T>
__device__ __forceinline__ void heat_body(const VB vb, const StepConsts& K, const Dev& d, const ParticleSoA<T>& PA,
                                          const ParticleSoA<T>& PB)
{
    const ParticleSoA<T> A = *d.bufsel ? PB : PA;
    const int n = d.counts[0];
    const T sc[9] = {T(pow2(K.fx0)), T(pow2(K.fx1)), T(pow2(K.fx1)), T(pow2(K.fx_s2)),
                     T(pow2(K.fx_s2)), T(pow2(K.fx_s2)), T(pow2(K.fx_s2)), T(pow2(K.fx_s3)),
                     T(pow2(K.fx_s3))};
    unsigned long long* h = reinterpret_cast<unsigned long long*>(d.whq);
    for (int i = vb.b * blockDim.x + threadIdx.x; i < n; i += vb.n * blockDim.x) {
        const int ci = A.cell[i];
        if (ci < 0) continue;   // a hole
        const T m = A.m[i], u = A.u[i], v = A.v[i], w = A.w[i];
        const T q = (u * u + v * v) + w * w;
        const T mu = m * u, mv = m * v;
        const T val[9] = {m, mu, mv, mu * u, mu * v, mv * v, m * q, mu * q, mv * q};
        const size_t c = (size_t)ci;
#pragma unroll
        for (int k = 0; k < 9; ++k) atomicAdd(h + 9 * c + k, (unsigned long long)fixp(val[k], sc[k], d.err));
    }
}
template <typename T>
__global__ void __launch_bounds__(256) k_heat_tally(const StepConsts K, const Dev d, ParticleSoA<T> PA, ParticleSoA<T> PB)
{
    heat_body<T>(UGKWP_VB_LAUNCH, K, d, PA, PB);
}

// ----------------------------------------------------- a2: new collisionless particles (Eq. 26)
// One thread per new particle over the step's flat range of new particles (cell c's N^hp particles take the
// slots nhp_off[c] .. nhp_off[c] + N^hp - 1 after the retained ones, in cell order); a thread finds its cell by
// a binary search of the exclusive scan nhp_off. Velocities are independent draws from the local distribution
// of the cell at U_i, T_i (Sec. III B): U_i + sqrt(R T_i) z with z Box-Muller normals (Pr = 1) or from the
// Shakhov acceptance-rejection (Pr != 1); no per-cell moment matching (forcing a few particles onto the cell's
// exact momentum and energy changes their speed distribution, and with it the speed-weighted fluxes such as the
// energy carried to a wall). W^{p,-} and W^{p,+} of the new particles: per warp, sums over each run of lanes
// holding the same cell (a segmented scan by shuffles), one 64-bit atomic add per run and moment.
template <typename T>
__device__ __forceinline__ void sample_body(const VB vb, const StepConsts& K, const Dev& d, const ParticleSoA<T>& PA,
                                            const ParticleSoA<T>& PB, const PCell<T>& pc, const long long* dstep)
{
    const ParticleSoA<T> A = *d.bufsel ? PB : PA;   // the buffer holding this step's particles
    const int total = d.counts[1];
    if (total == 0) return;
    const int nret = d.counts[0];
    const int room = d.counts[3] - nret;
    const int lane = threadIdx.x & 31;
    const Rng g{K.k0, K.k1, (uint32_t)*dstep};
    const uint64_t step_hi = (uint64_t)(uint32_t)*dstep << 32;
    const T s0 = T(pow2(K.fx0)), s1 = T(pow2(K.fx1)), s4 = T(pow2(K.fx4));
    int fallbacks = 0;
    const int stride = vb.n * blockDim.x;
    for (int k0 = vb.b * blockDim.x + (threadIdx.x & ~31); k0 < total; k0 += stride) {
        const int k = k0 + lane;
        int c = -1;
        long long acc[5] = {0, 0, 0, 0, 0};
        if (k < total) {
            // the last cell whose range starts at or before k (nhp_off[C] read as the total)
            int lo = 0, hi = K.C;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(d.nhp_off + mid) <= k) lo = mid;
                else hi = mid;
            }
            c = lo;
        }
        if (k < total && k >= room) {
            atomicOr(d.err, ERR_CAPACITY);
        } else if (k < total) {
            const int kl = k - __ldg(d.nhp_off + c);
            const uint64_t pid = step_hi | ((uint64_t)c << 11) | (uint64_t)kl;
            // Pr = 1: Box-Muller normals. Pr != 1: the Shakhov g^S of Eq. 4 by acceptance-rejection (Sec. III B):
            // Maxwellian proposals accepted with probability (1 + psi) / M, psi = (a . z)(|z|^2 - 5), |z| > 6
            // rejected; after kArAttempts rejections the last proposal stays
            T z0 = 0, z1 = 0, z2 = 0;
            const T ax = K.shakhov ? pc.q_(c, 0) : T(0), ay = K.shakhov ? pc.q_(c, 1) : T(0);
            const T M = K.shakhov ? pc.q_(c, 2) : T(1);
            const int attempts = K.shakhov ? kArAttempts : 1;
            bool accepted = !K.shakhov;
            for (int a = 0; a < attempts; ++a) {
                T U[4];
                Unif<T>::get(g, pid, K.shakhov ? draw_ar(a) : DRAW_VEL, 4, U);
                const T r0 = fsqrt_(T(-2) * dlog(U[0]));
                T sn0, cs0, sn1, cs1;
                dsincos2pi(U[1], &sn0, &cs0);
                const T r1 = fsqrt_(T(-2) * dlog(U[2]));
                dsincos2pi(U[3], &sn1, &cs1);
                z0 = r0 * cs0; z1 = r0 * sn0; z2 = r1 * cs1;
                if (!K.shakhov) break;
                const T s2 = (z0 * z0 + z1 * z1) + z2 * z2;
                if (s2 <= T(36)) {
                    const T psi = (z0 * ax + z1 * ay) * (s2 - T(5));
                    T Ua[1];
                    Unif<T>::get(g, pid, draw_ar(a) + 2u, 1, Ua);
                    if (Ua[0] * M < T(1) + psi) { accepted = true; break; }
                }
            }
            if (!accepted) fallbacks++;
            // uniform position: 1-D on the segment; 2-D the quad split along its 0-2 diagonal, a triangle chosen
            // by area, then barycentric (sqrt(U1), U2)
            T X[4], Y[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                X[q] = T(d.cvx[4 * c + q]);
                Y[q] = K.dim == 1 ? T(0) : T(d.cvy[4 * c + q]);
            }
            T U[3], x, y;
            Unif<T>::get(g, pid, DRAW_POS, 3, U);
            if (K.dim == 1) {
                x = X[0] + U[0] * (X[1] - X[0]);
                y = T(0);
            } else {
                const T A1 = T(0.5) * ((X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]));
                const T A2 = T(0.5) * ((X[2] - X[0]) * (Y[3] - Y[0]) - (X[3] - X[0]) * (Y[2] - Y[0]));
                const bool first = U[0] * (A1 + A2) < A1;
                const int bi = first ? 1 : 2, ci = first ? 2 : 3;
                const T sq = fsqrt_(U[1]);
                const T wa = T(1) - sq, wb = sq * (T(1) - U[2]), wc = sq * U[2];
                x = (wa * X[0] + wb * X[bi]) + wc * X[ci];
                y = (wa * Y[0] + wb * Y[bi]) + wc * Y[ci];
            }
            const T sig = fsqrt_(pc.s_(c, 2));
            const T un = pc.s_(c, 0) + sig * z0, vn = pc.s_(c, 1) + sig * z1, wn = sig * z2;
            const T m = pc.m_(c);
            const long long i = (long long)nret + k;
            A.x[i] = x; A.y[i] = y;
            A.u[i] = un;
            A.v[i] = vn;
            A.w[i] = wn;
            A.m[i] = m;
            A.cell[i] = c;
            A.pid[i] = pid;
            fix5(m, un, vn, wn, s0, s1, s4, d.err, acc);
        }
        // runs of lanes holding the same cell are contiguous: inclusive segmented sums, then the run's last lane
        // adds them to W^{p,-} and W^{p,+} (atomic: a cell's particles can span warps; W^{p,+} also takes the
        // ghost sources' particles on the second stream)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int co = __shfl_up_sync(0xffffffffu, c, o);
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const long long v = __shfl_up_sync(0xffffffffu, acc[q], o);
                if (lane >= o && co == c) acc[q] += v;
            }
        }
        const int cn = __shfl_down_sync(0xffffffffu, c, 1);
        if (c >= 0 && (lane == 31 || cn != c))
            for (int q = 0; q < 5; ++q)
                if (acc[q]) {
                    atomicAdd(reinterpret_cast<unsigned long long*>(d.wm) + 5 * (size_t)c + q, (unsigned long long)acc[q]);
                    atomicAdd(reinterpret_cast<unsigned long long*>(d.wpl) + 5 * (size_t)c + q, (unsigned long long)acc[q]);
                }
    }
    if (K.shakhov) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fallbacks += __shfl_xor_sync(0xffffffffu, fallbacks, o);
        if (lane == 0 && fallbacks) atomicAdd(d.stats + 12, (unsigned long long)fallbacks);
    }
}
template <typename T>
__global__ void __launch_bounds__(128) k_sample(const StepConsts K, const Dev d, ParticleSoA<T> PA,
                                                ParticleSoA<T> PB, PCell<T> pc, const long long* dstep)
{
    sample_body<T>(UGKWP_VB_LAUNCH, K, d, PA, PB, pc, dstep);
}

// A cell's outward normals and plane offsets (the stay and exit tests), copied into registers by 16-byte loads
// issued together: one memory round trip per cell visited
template <typename T> struct FaceGeo { T nx[4], ny[4], d[4]; };
template <typename T>
__device__ __forceinline__ FaceGeo<T> load_geo(const CellFaces<T>* __restrict__ cf, int c)
{
    constexpr int nw = sizeof(FaceGeo<T>) / 16;
    static_assert(sizeof(FaceGeo<T>) % 16 == 0, "normals and offsets of whole 16-byte words");
    const uint4* src = reinterpret_cast<const uint4*>(cf + c);
    uint4 w[nw];
#pragma unroll
    for (int k = 0; k < nw; ++k) w[k] = __ldg(src + k);
    FaceGeo<T> G;
    memcpy(&G, w, sizeof G);
    return G;
}

// A particle at (x, y) moving with (u, v) stays in its cell for the time tr when it reaches none of the faces
// ahead (n_k . u > 0; the face `entry` is skipped): tr (n_k . u) <= d_k - n_k . x for each of them. No
// division on this path, which almost every particle takes.
template <typename T>
__device__ __forceinline__ bool stays_in(const FaceGeo<T>& F, int nf, int entry, T x, T y, T u, T v, T tr)
{
    bool stays = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k >= nf || k == entry) continue;
        const T un = F.nx[k] * u + F.ny[k] * v;
        if (!(un > T(0))) continue;
        if (tr * un > F.d[k] - (F.nx[k] * x + F.ny[k] * y)) stays = false;
    }
    return stays;
}

// stays_in for the first transport test of a particle in its start cell (no entry face), FP32: the cell's
// outward normals and plane offsets in three 16-byte loads and the faces unrolled (faces past nf skipped), the
// same per-face operations as stays_in
__device__ __forceinline__ bool stays_in_start(const CellFaces<float>& F, int nf, float x, float y, float u, float v,
                                               float tr)
{
    const float4 NX = *reinterpret_cast<const float4*>(F.nx);
    const float4 NY = *reinterpret_cast<const float4*>(F.ny);
    const float4 D = *reinterpret_cast<const float4*>(F.d);
    const float nxa[4] = {NX.x, NX.y, NX.z, NX.w}, nya[4] = {NY.x, NY.y, NY.z, NY.w}, da[4] = {D.x, D.y, D.z, D.w};
    bool stays = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float un = nxa[k] * u + nya[k] * v;
        const bool ahead = k < nf && un > 0.0f;
        if (ahead && tr * un > da[k] - (nxa[k] * x + nya[k] * y)) stays = false;
    }
    return stays;
}

// The face through which a particle at (x, y) moving with (u, v) leaves its cell first: exit time through face
// k = (d_k - n_k . x) / (n_k . u) for n_k . u > 0 (negative values, from rounding on a face, count as 0); the
// smallest wins, ties go to the lower local index; the face `entry` is skipped. Returns the local index, or -1
// when no face lies ahead, and the exit time in best. Called when stays_in is false, so a face lies ahead.
template <typename T>
__device__ __forceinline__ int first_exit(const FaceGeo<T>& F, int nf, int entry, T x, T y, T u, T v, T& best)
{
    int kb = -1;
    best = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k >= nf || k == entry) continue;
        const T un = F.nx[k] * u + F.ny[k] * v;
        if (!(un > T(0))) continue;
        T t = (F.d[k] - (F.nx[k] * x + F.ny[k] * y)) / un;
        if (t < T(0)) t = T(0);
        if (kb < 0 || t < best) { best = t; kb = k; }
    }
    return kb;
}

// Free flight of one particle for the time tr left from cell c (the face `entry` excluded from the first exit
// test: the face it came in through, or -1): exit time through the cell's faces; at a crossing L -> R the
// mass and the remaining time scale by dt_R / dt_L (Eqs. 41, 52); diffuse re-emission at walls (wall tallies),
// specular mirrors, deletion at far-field and fixed ghosts. Returns alive; c is the final cell, it the number
// of face events.
template <typename T>
__device__ __forceinline__ bool fly(const Dev& d, const CellFaces<T>* __restrict__ cf, const Rng& g, T s0, T s1, T s4,
                                    T m2RTw, T sigw, T ws, T& x, T& y, T& u, T& v, T& w, T& m, T tr, int& c, int entry,
                                    uint64_t pid, int& it, unsigned long long& n_cross, unsigned long long& n_hits)
{
    int hits = 0;
    it = 0;
    bool alive = true;
    for (;;) {
        const FaceGeo<T> G = load_geo(cf, c);
        const int nf = d.nfc[c];
        if (stays_in(G, nf, entry, x, y, u, v, tr)) {
            x = x + u * tr;
            y = y + v * tr;
            break;
        }
        T best;
        const int kb = first_exit(G, nf, entry, x, y, u, v, best);
        const CellFaces<T>& F = cf[c];   // the exit face's data (in L1: the same lines as the normals)
        if (best > tr) best = tr;
        x = x + u * best;
        y = y + v * best;
        tr = tr - best;
        if (++it > kMaxIters) { atomicOr(d.err, ERR_LIMIT); break; }
        const int meta = F.meta[kb];
        const int bc = (meta >> 26) & 7;
        const int nb = F.nbr[kb];
        if (nb >= 0) {
            const int f = meta & 0xffffff, dir = ((meta >> 29) & 1) ? 0 : 1;
            atomicAdd(d.cross + 2 * f + dir, 1u);
            n_cross++;
            const T r = F.ratio[kb];
            // record mode (S33): the crossing mass before and after the scaling, fixed point of the mass exponent
            unsigned long long* rec = d.frec ? reinterpret_cast<unsigned long long*>(d.frec) + 4 * (size_t)f + 2 * dir
                                             : nullptr;
            if (rec) atomicAdd(rec, (unsigned long long)fixp(m, s0, d.err));
            m = m * r;
            tr = tr * r;
            if (rec) atomicAdd(rec + 1, (unsigned long long)fixp(m, s0, d.err));
            if (bc == UGKWP_BC_PERIODIC) x = x + T(d.cshift[4 * c + kb]);
            entry = (meta >> 24) & 3;
            c = nb;
        } else if (bc == UGKWP_BC_WALL) {
            // Maxwell wall: specular reflection with probability ws (the hit's fourth uniform), else diffuse
            // re-emission at T_w
            T U[4];
            Unif<T>::get(g, pid, draw_wall(hits), 4, U);
            const T nx = F.nx[kb], ny = F.ny[kb];
            T uo, vo, wz;
            if (ws > T(0) && U[3] < ws) {
                const T t2 = T(2) * (nx * u + ny * v);
                uo = u - t2 * nx;
                vo = v - t2 * ny;
                wz = w;
            } else {
                const T un = fsqrt_(m2RTw * dlog(U[0]));
                const T rad = fsqrt_(T(-2) * dlog(U[1]));
                T sn, cs;
                dsincos2pi(U[2], &sn, &cs);
                const T vt = sigw * (rad * cs);
                const T tx = -ny, ty = nx;
                wz = sigw * (rad * sn);
                uo = vt * tx - un * nx;
                vo = vt * ty - un * ny;
            }
            const int iw = d.fwall[meta & 0xffffff];
            const T ein = T(0.5) * ((u * u + v * v) + w * w);
            const T eout = T(0.5) * ((uo * uo + vo * vo) + wz * wz);
            unsigned long long* wa = reinterpret_cast<unsigned long long*>(d.wallt + 3 * (size_t)iw);
            atomicAdd(wa + 0, (unsigned long long)fixp(m * (u - uo), s1, d.err));
            atomicAdd(wa + 1, (unsigned long long)fixp(m * (v - vo), s1, d.err));
            atomicAdd(wa + 2, (unsigned long long)fixp(m * (ein - eout), s4, d.err));
            u = uo; v = vo; w = wz;
            entry = kb;
            hits++;
            n_hits++;
        } else if (bc == UGKWP_BC_SYMMETRY) {
            const T un = F.nx[kb] * u + F.ny[kb] * v;
            const T t2 = T(2) * un;
            u = u - t2 * F.nx[kb];
            v = v - t2 * F.ny[kb];
            entry = kb;
        } else {
            alive = false;
            break;
        }
    }
    return alive;
}

// W^{p,+} started as W^{p,-} (each particle unchanged in its cell). A particle that crossed a face, met a
// boundary or left moves its contribution; a collided one that stays is added to wcol, and the retained tally
// W^{p,+} - wcol is formed in k_update. Integer sums: identical to summing every final contribution.
template <typename T>
__device__ __forceinline__ void tally_move(const Dev& d, T s0, T s1, T s4, int it, bool alive, bool collide, int c0,
                                           T m0, T u0, T v0, T w0, int c, T m, T u, T v, T w)
{
    unsigned long long* pl = reinterpret_cast<unsigned long long*>(d.wpl);
    unsigned long long* cl = reinterpret_cast<unsigned long long*>(d.wcol);
    if (it > 0) {
        long long o[5], f[5];
        fix5(m0, u0, v0, w0, s0, s1, s4, d.err, o);
        if (alive) fix5(m, u, v, w, s0, s1, s4, d.err, f);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            atomicAdd(pl + 5 * (size_t)c0 + k, (unsigned long long)(-o[k]));
            if (alive) atomicAdd(pl + 5 * (size_t)c + k, (unsigned long long)f[k]);
            if (alive && collide) atomicAdd(cl + 5 * (size_t)c + k, (unsigned long long)f[k]);
        }
    } else if (collide) {
        long long o[5];
        fix5(m0, u0, v0, w0, s0, s1, s4, d.err, o);
#pragma unroll
        for (int k = 0; k < 5; ++k) atomicAdd(cl + 5 * (size_t)c0 + k, (unsigned long long)o[k]);
    }
}

// Survivors per cell for the counting sort (sort steps only): one atomic per run of equal cell in the warp
// (key -1: no survivor in this lane). Every lane of the warp takes part.
__device__ __forceinline__ void count_runs(const Dev& d, int key)
{
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    int start = (lane == 0 || prev != key) ? lane : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, start, o);
        if (lane >= o) start = max(start, t);
    }
    const int nx = __shfl_down_sync(0xffffffffu, key, 1);
    if ((lane == 31 || nx != key) && key >= 0) atomicAdd(d.cnt + key, lane - start + 1);
}

// A particle's record after transport, in place (slot i of the buffer that holds the step's particles): one
// that stayed in its start cell without a face event and without colliding has only moved (x, y written back);
// one that crossed or met a boundary writes its whole record but its id; a removed one (collided, or left the
// domain) becomes a hole (cell -1), squeezed out by the next counting sort.
template <typename T>
__device__ __forceinline__ void write_in_place(const ParticleSoA<T>& A, int i, bool moved_only, bool kept, T x, T y,
                                               T u, T v, T w, T m, int c)
{
    if (!kept) {
        A.cell[i] = -1;
        return;
    }
    A.x[i] = x; A.y[i] = y;
    if (!moved_only) {
        A.u[i] = u; A.v[i] = v; A.w[i] = w; A.m[i] = m;
        A.cell[i] = c;
    }
}

// ------------------------------------------------- a3-a6: free flight, transport and tallies
// One thread per particle (warp-uniform grid-stride loop). Retained particles draw t_f (Eq. 27 with dt_i),
// new ones fly the whole dt_i; free transport through the cell faces (Eq. 28) with mass and remaining time
// scaled by dt_R / dt_L at every crossing (Eqs. 41, 52), diffuse re-emission at walls, specular mirrors,
// deletion at far-field and fixed ghosts. Then W^{p,+} and the retained tally, and the particle's record in
// place (holes, cell -1, are skipped); on sort steps the survivors per cell for the counting sort.
template <typename T>
__global__ void __launch_bounds__(256, UGKWP_PARTICLES_MINB) k_particles(const StepConsts K, const Dev d, ParticleSoA<T> PA,
                                                   ParticleSoA<T> PB, const CellFaces<T>* __restrict__ cf,
                                                   PCell<T> pc, const long long* dstep)
{
    const ParticleSoA<T> A = *d.bufsel ? PB : PA;
    const bool sort_step = d.flags[0] != 0;
    const int nret = d.counts[0];
    const int n = nret + d.counts[1];
    const Rng g{K.k0, K.k1, (uint32_t)*dstep};
    const T s0 = T(pow2(K.fx0)), s1 = T(pow2(K.fx1)), s4 = T(pow2(K.fx4));
    const T m2RTw = T(K.m2RTw), sigw = T(K.sig_w);
    unsigned long long n_cross = 0, n_hits = 0, n_removed = 0, n_left = 0, n_kept = 0;
    int max_it = 0;
    const int lane = threadIdx.x & 31;
    // each warp takes chunks of K.chunk consecutive particles (of the cell-ordered array) from a global
    // counter and walks them 32 at a time, prefetching the next 32 records into L1 while it works on the
    // current ones; dynamic chunks keep all SMs busy when other kernels share the GPU
    for (;;) {
    int wbeg = 0;
    if (lane == 0) wbeg = atomicAdd(d.counts + 5, K.chunk);
    wbeg = __shfl_sync(0xffffffffu, wbeg, 0);
    if (wbeg >= n) break;
    const int wend = min(n, wbeg + K.chunk);
    for (int base = wbeg; base < wend; base += 32) {
        const int i = base + lane;
        const int inext = i + 32;
        if (inext < wend) {
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.x + inext));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.y + inext));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.u + inext));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.v + inext));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.cell + inext));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.pid + inext));
        }
        int end_cell = -1;
        bool kept = false;
        int c = i < wend ? A.cell[i] : -1;
        if (c >= 0) {
            T x = A.x[i], y = A.y[i], u = A.u[i], v = A.v[i], w = A.w[i], m = A.m[i];
            const uint64_t pid = A.pid[i];
            const int c0 = c;
            const T m0 = m, u0 = u, v0 = v, w0 = w;
            const T dtc = pc.dt_(c);
            T tr;
            bool collide = false;
            if (i >= nret) {
                tr = dtc;
            } else {
                // Eq. 27: t_f = -tau_i ln eps falls short of dt_i exactly when eps > e^{-dt_i / tau_i}; the
                // logarithm only for the colliding particles (t_f capped at dt_i against rounding)
                T U[1];
                Unif<T>::get(g, pid, DRAW_TF, 1, U);
                collide = U[0] > pc.emx_(c);
                tr = dtc;
                if (collide) {
                    const T a = -(pc.tau_(c) * dlog(U[0]));
                    if (a < dtc) tr = a;
                }
            }
            int it = 0;
            const bool alive = fly(d, cf, g, s0, s1, s4, m2RTw, sigw, T(K.wall_specular), x, y, u, v, w, m, tr, c, -1, pid, it,
                                   n_cross, n_hits);
            max_it = max(max_it, it);
            if (alive) {
                end_cell = c;
                kept = !collide;
                if (collide) n_removed++;
            } else {
                n_left++;
            }
            tally_move(d, s0, s1, s4, it, alive, collide, c0, m0, u0, v0, w0, c, m, u, v, w);
            write_in_place(A, i, it == 0 && !collide, kept, x, y, u, v, w, m, c);
            n_kept += kept ? 1 : 0;
        }
        if (sort_step) count_runs(d, kept ? end_cell : -1);
    }
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_cross += __shfl_xor_sync(0xffffffffu, n_cross, o);
        n_hits += __shfl_xor_sync(0xffffffffu, n_hits, o);
        n_removed += __shfl_xor_sync(0xffffffffu, n_removed, o);
        n_left += __shfl_xor_sync(0xffffffffu, n_left, o);
        n_kept += __shfl_xor_sync(0xffffffffu, n_kept, o);
        max_it = max(max_it, __shfl_xor_sync(0xffffffffu, max_it, o));
    }
    if (lane == 0) {
        if (n_removed) atomicAdd(d.stats + 3, n_removed);
        if (n_left) atomicAdd(d.stats + 4, n_left);
        if (n_cross) atomicAdd(d.stats + 5, n_cross);
        if (n_hits) atomicAdd(d.stats + 6, n_hits);
        if (max_it) atomicMax(d.stats + 7, (unsigned long long)max_it);
        if (n_kept) atomicAdd(d.counts + 2, (int)n_kept);
    }
}

// ---------------------------------------- bulk asynchronous copies into shared memory, with mbarriers
constexpr unsigned long long kCopyWaitNs = 2000000000ull;   // bounded wait for a tile's copies (2 s)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// waits for the phase of the given parity with a time limit; false when the limit ran out
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u && global_ns() - t0 > kCopyWaitNs) return false;
    }
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// ---------------------------------------- a3-a7, warp-staged: the production-precision transport kernels
// Two passes. The stay pass (k_particles_warp): every warp works alone (no block-wide barrier); it claims
// tiles of WT consecutive particle slots from a global counter and has the fields that the stay test reads
// (cell, x, y, u, v, id) copied into its own shared memory by bulk asynchronous copies (cp.async.bulk,
// completion counted on the warp's mbarrier), double-buffered, so that the next tile streams in while the
// warp works on the current one. Per particle: t_f (Eq. 27, computed form as in k_particles) and the stay test
// of the start cell, 32 particles at a time with no warp-wide operation between them (their loads and Philox
// chains overlap). A particle that stays and does not collide has only moved: its x, y are written back in
// place (8 bytes), the rest of its record is left untouched. Holes (cell -1) are skipped. The others (a face
// ahead within t_r, or colliding; a few percent) go to a global queue: slot, t_r, collide and the fields the
// warp holds, so that the flight pass reads them contiguously and gathers only w and m.
// The flight pass (k_particles_fly): one thread per queued particle, at full occupancy and with nothing else
// waiting on it: the full free flight of fly() (crossings with the dt_R / dt_L scaling, walls, exits) and the
// tallies, exactly as in k_particles, then the record in place (the whole record but the id, or a hole).
// On sort steps the survivors are counted per cell for the counting sort. Every per-particle operation is
// that of k_particles, in the same order, so the results are identical.
constexpr int kWWarps = 4;     // warps per CTA of the stay pass

template <int WT> struct alignas(16) WarpSmem {
    float x[2][WT], y[2][WT], u[2][WT], v[2][WT];   // two stages of tile fields
    int cell[2][WT];
    unsigned long long pid[2][WT];
    unsigned long long bar[2];
};

// lane 0: copy the stay-test fields of tile t of A into stage b of the warp's shared memory (the slot count
// rounded up to 4, which the buffers' slack covers, so that every copy is a multiple of 16 bytes from a
// 16-byte aligned address)
template <int WT>
__device__ __forceinline__ void wtile_issue(const ParticleSoA<float>& A, int t, int n, WarpSmem<WT>& S, int b)
{
    const int base = t * WT;
    const int cnt4 = (min(WT, n - base) + 3) & ~3;
    const uint32_t b4 = (uint32_t)cnt4 * 4u, b8 = (uint32_t)cnt4 * 8u;
    unsigned long long* bar = &S.bar[b];
    mbar_expect_tx(bar, 5u * b4 + b8);
    bulk_load(S.x[b], A.x + base, b4, bar);
    bulk_load(S.y[b], A.y + base, b4, bar);
    bulk_load(S.u[b], A.u + base, b4, bar);
    bulk_load(S.v[b], A.v + base, b4, bar);
    bulk_load(S.cell[b], A.cell + base, b4, bar);
    bulk_load(S.pid[b], A.pid + base, b8, bar);
}

// false when a tile's copies did not arrive in time (ERR_LIMIT set; the copies in flight were given their own
// bounded wait)
template <int WT>
__device__ __forceinline__ bool stay_body(const StepConsts& K, const Dev& d, const ParticleSoA<float>& PA,
                                          const ParticleSoA<float>& PB, const CellFaces<float>* __restrict__ cf,
                                          const long long* dstep)
{
    extern __shared__ __align__(128) unsigned char warp_smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem<WT>& S = reinterpret_cast<WarpSmem<WT>*>(warp_smem_raw)[wid];
    const ParticleSoA<float> A = *d.bufsel ? PB : PA;
    const bool sort_step = d.flags[0] != 0;
    const int nret = d.counts[0];
    const int n = nret + d.counts[1];
    const int ntiles = (n + WT - 1) / WT;
    const Rng g{K.k0, K.k1, (uint32_t)*dstep};
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned long long n_kept = 0;

    if (lane == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // tiles are claimed one ahead of the copies: the claim of the tile after next is in flight while the warp
    // works, so its latency is hidden (lane 0 holds the claims)
    int tile = 0, ahead = 0;
    if (lane == 0) {
        tile = atomicAdd(d.counts + 5, 1);
        ahead = atomicAdd(d.counts + 5, 1);
        if (tile < ntiles) wtile_issue<WT>(A, tile, n, S, 0);
    }
    tile = __shfl_sync(0xffffffffu, tile, 0);
    int b = 0;
    uint32_t parity[2] = {0u, 0u};
    uint32_t pending = tile < ntiles ? 1u : 0u;   // stages with copies in flight (bit per stage)
    bool abort = false;
    while (tile < ntiles) {
        // start the next tile's copies into the other stage (released at the end of the last tile), claim the
        // one after
        const int nxt = __shfl_sync(0xffffffffu, ahead, 0);
        if (lane == 0 && nxt < ntiles) {
            wtile_issue<WT>(A, nxt, n, S, b ^ 1);
            ahead = atomicAdd(d.counts + 5, 1);
        }
        if (nxt < ntiles) pending |= 1u << (b ^ 1);
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&S.bar[b], parity[b]))) {
            abort = true;
            break;
        }
        parity[b] ^= 1u;
        pending &= ~(1u << b);
        const int base = tile * WT, cnt = min(WT, n - base);

        // t_f and the stay test of the start cell for the whole tile; particles that only move are done, the
        // others are queued for the flight pass
        int code[WT / 32];      // 0 hole, 1 moved only, 2 queued, 3 queued and colliding
        float trq[WT / 32];
#pragma unroll
        for (int r = 0; r < WT / 32; ++r) {
            const int j = r * 32 + lane;
            const int c = j < cnt ? S.cell[b][j] : -1;
            code[r] = 0;
            trq[r] = 0.0f;
            if (c >= 0) {
                const int i = base + j;
                const float4 cd = d.cst32[c];   // dt, e^{-x}, tau, face count
                const float x = S.x[b][j], y = S.y[b][j], u = S.u[b][j], v = S.v[b][j];
                const float dtc = cd.x;
                float tr = dtc;
                bool collide = false;
                if (i < nret) {
                    float U[1];
                    Unif<float>::get(g, S.pid[b][j], DRAW_TF, 1, U);
                    collide = U[0] > cd.y;
                    if (collide) {
                        const float a = -(cd.z * dlog(U[0]));
                        if (a < dtc) tr = a;
                    }
                }
                const bool stays = stays_in_start(cf[c], __float_as_int(cd.w), x, y, u, v, tr);
                if (stays && !collide) {
                    A.x[i] = x + u * tr;
                    A.y[i] = y + v * tr;
                    code[r] = 1;
                    n_kept++;
                } else {
                    trq[r] = tr;
                    code[r] = collide ? 3 : 2;
                }
            }
        }
        // the queued particles of the tile: one slot range of the global queue per tile
        unsigned qm[WT / 32];
        int tot = 0;
#pragma unroll
        for (int r = 0; r < WT / 32; ++r) {
            qm[r] = __ballot_sync(0xffffffffu, code[r] >= 2);
            tot += __popc(qm[r]);
        }
        if (tot) {
            int qb = 0;
            if (lane == 0) qb = atomicAdd(d.nxq, tot);
            qb = __shfl_sync(0xffffffffu, qb, 0);
#pragma unroll
            for (int r = 0; r < WT / 32; ++r) {
                if (code[r] >= 2) {
                    const int e = qb + __popc(qm[r] & lt_mask), j = r * 32 + lane;
                    d.xq_i[e] = (base + j) | (code[r] == 3 ? (int)0x80000000u : 0);
                    d.xq_t[e] = trq[r];
                    d.xq.x[e] = S.x[b][j]; d.xq.y[e] = S.y[b][j]; d.xq.u[e] = S.u[b][j]; d.xq.v[e] = S.v[b][j];
                    d.xq.cell[e] = S.cell[b][j]; d.xq.pid[e] = S.pid[b][j];
                }
                qb += __popc(qm[r]);
            }
        }
        // sort steps: the tile's particles that only moved, per cell (the queued ones count when they fly)
        if (sort_step) {
#pragma unroll
            for (int r = 0; r < WT / 32; ++r) {
                const int j = r * 32 + lane;
                count_runs(d, code[r] == 1 ? S.cell[b][j] : -1);
            }
        }
        // this lane's generic-proxy accesses of the stage come before the bulk copy that refills it (issued by
        // lane 0 at the top of the next iteration)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        tile = nxt;
        b ^= 1;
    }
    if (abort) {
        // a tile's copies did not arrive in time: report it, and give the copies still in flight their own
        // bounded wait before the warp's shared memory is released
        if (lane == 0) {
            atomicOr(d.err, ERR_LIMIT);
            for (int q = 0; q < 2; ++q)
                if (pending & (1u << q)) (void)mbar_wait_bounded(&S.bar[q], parity[q]);
        }
        return false;
    }
    for (int o = 16; o > 0; o >>= 1) n_kept += __shfl_xor_sync(0xffffffffu, n_kept, o);
    if (lane == 0) {
        if (n_kept) atomicAdd(d.counts + 2, (int)n_kept);
        // every copy has completed: the barriers are retired, so that the shared memory can hold new ones
        mbar_inval(&S.bar[0]);
        mbar_inval(&S.bar[1]);
    }
    __syncwarp();
    return true;
}
template <int WT, int MINB>
__global__ void __launch_bounds__(kWWarps * 32, MINB) k_particles_warp(const StepConsts K, const Dev d,
                                                                       ParticleSoA<float> PA, ParticleSoA<float> PB,
                                                                       const CellFaces<float>* __restrict__ cf,
                                                                       const long long* dstep)
{
    (void)stay_body<WT>(K, d, PA, PB, cf, dstep);
}

// the flight pass: the queued particles of the stay pass, one per thread (warp-uniform grid-stride loop)
__device__ __forceinline__ void fly_body(const VB vb, const StepConsts& K, const Dev& d, const ParticleSoA<float>& PA,
                                         const ParticleSoA<float>& PB, const CellFaces<float>* __restrict__ cf,
                                         const long long* dstep)
{
    const ParticleSoA<float> A = *d.bufsel ? PB : PA;
    const bool sort_step = d.flags[0] != 0;
    const int nq = *d.nxq;
    const Rng g{K.k0, K.k1, (uint32_t)*dstep};
    const float s0 = float(pow2(K.fx0)), s1 = float(pow2(K.fx1)), s4 = float(pow2(K.fx4));
    const float m2RTw = float(K.m2RTw), sigw = float(K.sig_w), ws = float(K.wall_specular);
    const int lane = threadIdx.x & 31;
    unsigned long long n_cross = 0, n_hits = 0, n_removed = 0, n_left = 0, n_kept = 0;
    int max_it = 0;
    const int stride = vb.n * blockDim.x;
    for (int e0 = vb.b * blockDim.x + (threadIdx.x & ~31); e0 < nq; e0 += stride) {
        const int e = e0 + lane;
        int c = -1;
        bool kept = false;
        if (e < nq) {
            const int code = d.xq_i[e];
            const int i = code & 0x7fffffff;
            const bool collide = code < 0;
            float x = d.xq.x[e], y = d.xq.y[e], u = d.xq.u[e], v = d.xq.v[e], w = A.w[i], m = A.m[i];
            c = d.xq.cell[e];
            const unsigned long long pid = d.xq.pid[e];
            const int c0 = c;
            const float m0 = m, u0 = u, v0 = v, w0 = w;
            int it = 0;
            const bool alive = fly(d, cf, g, s0, s1, s4, m2RTw, sigw, ws, x, y, u, v, w, m, d.xq_t[e], c, -1,
                                   (uint64_t)pid, it, n_cross, n_hits);
            max_it = max(max_it, it);
            if (alive) {
                if (collide) n_removed++;
            } else {
                n_left++;
            }
            tally_move(d, s0, s1, s4, it, alive, collide, c0, m0, u0, v0, w0, c, m, u, v, w);
            kept = alive && !collide;
            write_in_place(A, i, it == 0 && !collide, kept, x, y, u, v, w, m, c);
            n_kept += kept ? 1 : 0;
        }
        if (sort_step) count_runs(d, kept ? c : -1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_cross += __shfl_xor_sync(0xffffffffu, n_cross, o);
        n_hits += __shfl_xor_sync(0xffffffffu, n_hits, o);
        n_removed += __shfl_xor_sync(0xffffffffu, n_removed, o);
        n_left += __shfl_xor_sync(0xffffffffu, n_left, o);
        n_kept += __shfl_xor_sync(0xffffffffu, n_kept, o);
        max_it = max(max_it, __shfl_xor_sync(0xffffffffu, max_it, o));
    }
    if (lane == 0) {
        if (n_removed) atomicAdd(d.stats + 3, n_removed);
        if (n_left) atomicAdd(d.stats + 4, n_left);
        if (n_cross) atomicAdd(d.stats + 5, n_cross);
        if (n_hits) atomicAdd(d.stats + 6, n_hits);
        if (max_it) atomicMax(d.stats + 7, (unsigned long long)max_it);
        if (n_kept) atomicAdd(d.counts + 2, (int)n_kept);
    }
}
__global__ void __launch_bounds__(128, UGKWP_FLY_MINB) k_particles_fly(const StepConsts K, const Dev d, ParticleSoA<float> PA,
                                                       ParticleSoA<float> PB, const CellFaces<float>* __restrict__ cf,
                                                       const long long* dstep)
{
    fly_body(UGKWP_VB_LAUNCH, K, d, PA, PB, cf, dstep);
}

// ------------------------------------------------ ghost particle sources (far-field and fixed faces)
// The virtual ghost cell behind a far-field / fixed face holds the ghost state with the fluid cell's time step
// dt_L; its collisionless part e^{-x}, x = dt_L / tau_g, is sampled as particles in a slab of depth
// D = (max(W_0, 0) + 6 sqrt(RT_g)) dt_L behind the face (W_0 the ghost's inflow speed); those that reach the
// face within dt_L enter the fluid cell at a uniform point of the face and fly, collisionless, for the rest
// of the step. Per source: N = ceil(M / m_ref) particles (at most kMaxNew) of mass M / N, M = rho_g e^{-x} s D,
// m_ref = rho_g Omega_L / N_ref; the ghost's wave free-transport weight is then dbar_d - e^{-x}.

// per source, FP64 (one thread each): ghost state, sample count, mass, ghost velocity, sqrt(RT), slab depth
__device__ __forceinline__ void injp_body(const VB vb, const StepConsts& K, const Dev& d)
{
    const int j = vb.b * blockDim.x + threadIdx.x;
    if (j >= K.n_inj) return;
    const int f = d.inj_face[j], L = d.fL[f];
    const double* Wg;
    if (d.fbc[f] == UGKWP_BC_FIXED) {
        Wg = K.W_fix;
    } else {
        const double un_inf = K.W_inf[1] * d.fnx[f] + K.W_inf[2] * d.fny[f];
        Wg = un_inf < 0.0 ? K.W_inf : d.W + 4 * L;
    }
    const double rho = Wg[0], r = 1.0 / rho, U = Wg[1] * r, V = Wg[2] * r;
    const double RT = (Wg[3] * r - 0.5 * (U * U + V * V)) * (2.0 / 3.0);
    const double x = d.dt[L] / tau_of(K, Wg);
    const double e = dexp(-x);
    const double sig = sqrt(RT);
    const double W0 = -(U * d.fnx[f] + V * d.fny[f]);
    const double D = ((W0 > 0.0 ? W0 : 0.0) + 6.0 * sig) * d.dt[L];
    const double M = ((rho * e) * d.fs[f]) * D;
    int n = 0;
    if (M > 0.0) {
        const double q = ceil(M / ((rho * d.vol[L]) / (double)K.n_ref));
        n = q > (double)kMaxNew ? kMaxNew : (q < 1.0 ? 1 : (int)q);
    }
    d.inj_n[j] = n;
    double* P = d.inj_par + 5 * j;
    P[0] = n > 0 ? M / (double)n : 0.0;
    P[1] = U; P[2] = V; P[3] = sig; P[4] = D;
}
__global__ void k_inject_params(const StepConsts K, Dev d) { injp_body(UGKWP_VB_LAUNCH, K, d); }

// one warp per source: sample, enter, fly, tally W^{p,+}, write the survivors like the transport kernel
template <typename T>
__device__ __forceinline__ void inject_body(const VB vb, const StepConsts& K, const Dev& d, const ParticleSoA<T>& PA,
                                            const ParticleSoA<T>& PB, const CellFaces<T>* __restrict__ cf,
                                            const long long* dstep)
{
    const int j = (vb.b * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= K.n_inj) return;
    const int N = d.inj_n[j];
    if (N == 0) return;
    // the entering particles that survive are appended past the step's slots of the buffer that holds the
    // step's particles (the transport kernel updates slots below n in place meanwhile)
    const ParticleSoA<T> B = *d.bufsel ? PB : PA;
    const bool sort_step = d.flags[0] != 0;
    const int n = d.counts[4], cap = d.counts[3];
    const int f = d.inj_face[j], L = d.fL[f], kin = d.inj_k[j];
    const Rng g{K.k0, K.k1, (uint32_t)*dstep};
    const uint64_t base = ((uint64_t)(uint32_t)*dstep << 32) | ((uint64_t)(K.C + j) << 11);
    const T s0 = T(pow2(K.fx0)), s1 = T(pow2(K.fx1)), s4 = T(pow2(K.fx4));
    const T m2RTw = T(K.m2RTw), sigw = T(K.sig_w);
    const T nx = T(d.fnx[f]), ny = T(d.fny[f]);
    const double* P = d.inj_par + 5 * j;
    const T m0 = T(P[0]), Ug = T(P[1]), Vg = T(P[2]), sig = T(P[3]), D = T(P[4]);
    const T dtL = T(d.dt[L]);
    const T ax = T(d.fax[f]), ay = T(d.fay[f]), ex = T(d.fex[f]), ey = T(d.fey[f]);
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned long long n_cross = 0, n_hits = 0, n_left = 0, n_in = 0;
    int max_it = 0;
    unsigned long long* pl = reinterpret_cast<unsigned long long*>(d.wpl);
    for (int k0 = 0; k0 < N; k0 += 32) {
        const int k = k0 + lane;
        bool kept = false;
        int c = L;
        T x = 0, y = 0, u = 0, v = 0, w = 0, m = m0;
        const uint64_t pid = base | (uint64_t)k;
        if (k < N) {
            T Up[3], Uv[4];
            Unif<T>::get(g, pid, DRAW_POS, 3, Up);
            Unif<T>::get(g, pid, DRAW_VEL, 4, Uv);
            const T r0 = fsqrt_(T(-2) * dlog(Uv[0]));
            T sn0, cs0, sn1, cs1;
            dsincos2pi(Uv[1], &sn0, &cs0);
            const T r1 = fsqrt_(T(-2) * dlog(Uv[2]));
            dsincos2pi(Uv[3], &sn1, &cs1);
            u = Ug + sig * (r0 * cs0);
            v = Vg + sig * (r0 * sn0);
            w = sig * (r1 * cs1);
            const T un = nx * u + ny * v;
            if (un < T(0)) {
                const T tc = (Up[0] * D) / (-un);
                if (tc < dtL) {
                    n_in++;
                    x = ax + Up[1] * ex;
                    y = ay + Up[1] * ey;
                    int it = 0;
                    const bool alive = fly(d, cf, g, s0, s1, s4, m2RTw, sigw, T(K.wall_specular), x, y, u, v, w, m, dtL - tc, c, kin, pid, it,
                                           n_cross, n_hits);
                    max_it = max(max_it, it);
                    if (alive) {
                        kept = true;
                        long long fq[5];
                        fix5(m, u, v, w, s0, s1, s4, d.err, fq);
#pragma unroll
                        for (int q = 0; q < 5; ++q) atomicAdd(pl + 5 * (size_t)c + q, (unsigned long long)fq[q]);
                    } else {
                        n_left++;
                    }
                }
            }
        }
        // survivors: slots reserved past n; those at or beyond the capacity are not written (an error), and
        // the bookkeeping of k_update and k_scatter counts the reserved slots only up to the capacity, so that
        // no later kernel touches a slot past it
        const unsigned km = __ballot_sync(0xffffffffu, kept);
        if (!km) continue;
        int slot0 = 0;
        if (lane == 0) slot0 = atomicAdd(d.counts + 7, __popc(km));
        slot0 = __shfl_sync(0xffffffffu, slot0, 0);
        const int jj = n + slot0 + __popc(km & lt_mask);
        const bool stored = kept && jj < cap;
        if (kept && !stored) atomicOr(d.err, ERR_CAPACITY);
        if (stored) {
            B.x[jj] = x; B.y[jj] = y; B.u[jj] = u; B.v[jj] = v; B.w[jj] = w; B.m[jj] = m;
            B.cell[jj] = c;
            B.pid[jj] = pid;
            if (sort_step) atomicAdd(d.cnt + c, 1);
        }
        const unsigned sm = __ballot_sync(0xffffffffu, stored);
        if (lane == 0 && sm) atomicAdd(d.counts + 2, __popc(sm));
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_cross += __shfl_xor_sync(0xffffffffu, n_cross, o);
        n_hits += __shfl_xor_sync(0xffffffffu, n_hits, o);
        n_left += __shfl_xor_sync(0xffffffffu, n_left, o);
        n_in += __shfl_xor_sync(0xffffffffu, n_in, o);
        max_it = max(max_it, __shfl_xor_sync(0xffffffffu, max_it, o));
    }
    if (lane == 0) {
        if (n_left) atomicAdd(d.stats + 4, n_left);
        if (n_cross) atomicAdd(d.stats + 5, n_cross);
        if (n_hits) atomicAdd(d.stats + 6, n_hits);
        if (max_it) atomicMax(d.stats + 7, (unsigned long long)max_it);
        if (n_in) { atomicAdd(d.stats + 13, n_in); atomicAdd(d.counts + 6, (int)n_in); }
    }
}
template <typename T>
__global__ void __launch_bounds__(128) k_inject(const StepConsts K, const Dev d, ParticleSoA<T> PA, ParticleSoA<T> PB,
                                                const CellFaces<T>* __restrict__ cf, const long long* dstep)
{
    inject_body<T>(UGKWP_VB_LAUNCH, K, d, PA, PB, cf, dstep);
}

// --------------------------------------------------------------------- a7: counting sort
// sort steps only: counting sort of the survivors by cell (holes dropped), from the buffer that holds the
// step's particles into the other one, which becomes the current one at the end of the step
template <typename T>
__device__ __forceinline__ void scatter_body(const VB vb, const Dev& d, const ParticleSoA<T>& PA, const ParticleSoA<T>& PB)
{
    if (!d.flags[0]) return;
    const int sel = *d.bufsel;
    const ParticleSoA<T> A = sel ? PB : PA, B = sel ? PA : PB;
    // the step's slots, then those of particles that entered from ghosts (reserved slots up to the capacity)
    const int n = min(d.counts[4] + d.counts[7], d.counts[3]);
    const int lane = threadIdx.x & 31;
    const int stride = vb.n * blockDim.x;
    // warp-uniform loop; the slots of a run of equal cells in the warp (the particles stay grouped by cell
    // between sorts) are reserved with one atomic by the run's first lane
    for (int i0 = vb.b * blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
        const int i = i0 + lane;
        const int c = i < n ? A.cell[i] : -1;
        const int prev = __shfl_up_sync(0xffffffffu, c, 1);
        int start = (lane == 0 || prev != c) ? lane : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, start, o);
            if (lane >= o) start = max(start, t);
        }
        const int nx = __shfl_down_sync(0xffffffffu, c, 1);
        int end = (lane == 31 || nx != c) ? lane : 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_down_sync(0xffffffffu, end, o);
            if (lane + o < 32) end = min(end, t);
        }
        int base = 0;
        if (lane == start && c >= 0) base = atomicAdd(d.cur + c, end - start + 1);
        base = __shfl_sync(0xffffffffu, base, start);
        if (c < 0) continue;
        const int slot = d.off[c] + base + (lane - start);
        B.x[slot] = A.x[i]; B.y[slot] = A.y[i]; B.u[slot] = A.u[i]; B.v[slot] = A.v[i]; B.w[slot] = A.w[i];
        B.m[slot] = A.m[i]; B.cell[slot] = c; B.pid[slot] = A.pid[i];
    }
}
template <typename T>
__global__ void __launch_bounds__(256) k_scatter(const Dev d, ParticleSoA<T> PA, ParticleSoA<T> PB)
{
    scatter_body<T>(UGKWP_VB_LAUNCH, d, PA, PB);
}

// ---------------------------------------------------------------- a10: update (Eq. 53)
// Threads [0, C): conservative update of one cell, residual term, particle-mass-ratio EMA, vacuum floor.
// Threads [C, C + n_wall): wall pressure, shear stress and heat flux of one wall face (a11, Sec. V A).
// The last block to finish reduces the residual partials in block order and closes the step.
constexpr int kUpdateBlock = 128;
__device__ __forceinline__ void update_body(const VB vb, const StepConsts& K, const Dev& d, long long* dstep)
{
    const int t = vb.b * blockDim.x + threadIdx.x;
    double r2[4] = {0, 0, 0, 0};
    if (t < K.C) {
        const int c = t;
        const CellFaces<float>& Fc = d.cf32[c];
        double acc[4] = {0, 0, 0, 0};
        for (int k = 0; k < d.nfc[c]; ++k) {
            const int meta = Fc.meta[k];
            const int f = meta & 0xffffff;
            const bool isL = (meta >> 29) & 1;
            const double s = d.fs[f];
            // one fused multiply-add per term (B300's FP64 pipe is narrow); the sum stays FP64
            for (int q = 0; q < 4; ++q) {
                const double fq = d.flux[4 * (size_t)f + q];
                acc[q] = __fma_rn(isL ? fq : -fq, s, acc[q]);
            }
        }
        // FP64 throughout; the divisions by Omega_i and dt_i are multiplications by their reciprocals
        const double vol = d.vol[c], dt = d.dt[c], rvol = d.rcp[2 * c], rdt = d.rcp[2 * c + 1];
        const double coef = dt * rvol;
        const double sc[4] = {pow2(-K.fx0), pow2(-K.fx1), pow2(-K.fx1), pow2(-K.fx4)};
        const int tk[4] = {0, 1, 2, 4};
        double* W = d.W + 4 * c;
        double Wn[4];
        for (int q = 0; q < 4; ++q) {
            const long long dd = d.wpl[5 * c + tk[q]] - d.wm[5 * c + tk[q]];
            Wn[q] = (W[q] - coef * acc[q]) + ((double)dd * sc[q]) * rvol;
        }
        if (K.dim == 1) Wn[2] = 0.0;
        if (!isfinite(Wn[0]) || !isfinite(Wn[1]) || !isfinite(Wn[2]) || !isfinite(Wn[3])) atomicOr(d.err, ERR_NONPHYS);
        // realizability floor: statistical noise can leave the wave's share W - W^p of a cell negative and
        // drive the updated state out of the realizable set. Such a cell restarts from its particle content
        // W^{p,+} / Omega_i (the next step's W^h = W - W^p is then the collided particles' mass, not negative),
        // speed limited to U_cap, temperature clamped to [T_min, T_cap]; a cell without particles restarts from
        // the near-vacuum state at rest at T_inf
        if (!realizable(K, Wn)) {
            double P[4];
            for (int q = 0; q < 4; ++q) P[q] = ((double)d.wpl[5 * c + tk[q]] * sc[q]) * rvol;
            if (K.dim == 1) P[2] = 0.0;
            if (P[0] > kRhoFloor) {
                const double r = 1.0 / P[0];
                double U = P[1] * r, V = P[2] * r;
                double q2 = U * U + V * V;
                if (q2 > K.U_cap * K.U_cap) {
                    const double f = K.U_cap / sqrt(q2);
                    U = U * f;
                    V = V * f;
                    q2 = U * U + V * V;
                }
                double e = P[3] * r - 0.5 * q2;
                const double emin = (1.5 * kR) * K.T_min, emax = (1.5 * kR) * K.T_cap;
                if (!(e >= emin)) e = emin;
                if (e > emax) e = emax;
                Wn[0] = P[0]; Wn[1] = P[0] * U; Wn[2] = P[0] * V; Wn[3] = P[0] * (e + 0.5 * q2);
            } else {
                Wn[0] = kRhoFloor; Wn[1] = 0.0; Wn[2] = 0.0; Wn[3] = kRhoFloor * (1.5 * kR);
            }
            atomicAdd(d.stats + 11, 1ull);
        }
        for (int q = 0; q < 4; ++q) {
            const double r = (Wn[q] - W[q]) * rdt;
            r2[q] = vol * (r * r);
            W[q] = Wn[q];
        }
        // retained tally of this step (the next step's W^p): W^{p,+} minus the collided particles that stay
        for (int k = 0; k < 5; ++k) d.wrt[5 * c + k] = d.wpl[5 * c + k] - d.wcol[5 * c + k];
        // particle mass fraction chi^p and its EMA (a diagnostic: FP32 arithmetic)
        const float chi = (((float)d.wpl[5 * c] * (float)sc[0]) * (float)rvol) / (float)W[0];
        const float ce = (float)d.chi_ema[c];
        d.chi_ema[c] = *dstep == 0 ? chi : ce + (2.0f / 1001.0f) * (chi - ce);
    } else if (t < K.C + K.nwall) {
        const int iw = t - K.C;
        const int f = d.wall_face[iw], c = d.fL[f];
        const double nx = d.fnx[f], ny = d.fny[f], tx = -ny, ty = nx;
        const double* F = d.flux + 4 * (size_t)f;
        const double s1 = pow2(-K.fx1), s4 = pow2(-K.fx4);
        const double rsdt = 1.0 / (d.fs[f] * d.dt[c]);
        const double px = ((double)d.wallt[3 * iw] * s1) * rsdt;
        const double py = ((double)d.wallt[3 * iw + 1] * s1) * rsdt;
        const double pe = ((double)d.wallt[3 * iw + 2] * s4) * rsdt;
        const double p = (F[1] + px) * nx + (F[2] + py) * ny;
        const double tw = (F[1] + px) * tx + (F[2] + py) * ty;
        const double q = F[3] + pe;
        d.surf_last[3 * iw] = p; d.surf_last[3 * iw + 1] = tw; d.surf_last[3 * iw + 2] = q;
        d.surf_sum[3 * iw] += p; d.surf_sum[3 * iw + 1] += tw; d.surf_sum[3 * iw + 2] += q;
    }
    // residual partial sums in a fixed tree order
    __shared__ double sm[4][kUpdateBlock];
    __shared__ bool last;
    for (int q = 0; q < 4; ++q) sm[q][threadIdx.x] = r2[q];
    __syncthreads();
    for (int s = kUpdateBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int q = 0; q < 4; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; ++q) d.res_part[4 * vb.b + q] = sm[q][0];
        __threadfence();
        last = atomicAdd(d.done, 1u) == (unsigned)vb.n - 1u;
    }
    __syncthreads();
    if (!last) return;
    // the step's last block: residual (the block partials summed by all its threads in a fixed order: thread t
    // takes blocks t, t + 256, ..., then the same tree as above), counters, next step
    __threadfence();
    double s[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < vb.n; b += kUpdateBlock)
        for (int q = 0; q < 4; ++q) s[q] += __ldcg(d.res_part + 4 * b + q);
    for (int q = 0; q < 4; ++q) sm[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int h = kUpdateBlock / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int q = 0; q < 4; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + h];
        __syncthreads();
    }
    // monitored wall loads (Sec. V A, V B): F_x = sum_j s_j (p_j n_x - tau_j n_y), Q = sum_j s_j q_j over the
    // wall faces, summed by the block like the residual (thread t: faces t, t + 128, ..., then the tree)
    double fx = 0.0, fq = 0.0;
    for (int iw = threadIdx.x; iw < K.nwall; iw += kUpdateBlock) {
        const int f = d.wall_face[iw];
        const double* sv = d.surf_last + 3 * (size_t)iw;
        fx += d.fs[f] * (sv[0] * d.fnx[f] - sv[1] * d.fny[f]);
        fq += d.fs[f] * sv[2];
    }
    __syncthreads();
    const double rs0 = sm[0][0], rs1 = sm[1][0], rs2 = sm[2][0], rs3 = sm[3][0];
    __syncthreads();
    sm[0][threadIdx.x] = fx;
    sm[1][threadIdx.x] = fq;
    __syncthreads();
    for (int h = kUpdateBlock / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + h];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    d.res[0] = sqrt(rs0); d.res[1] = sqrt(rs1); d.res[2] = sqrt(rs2); d.res[3] = sqrt(rs3);
    {
        // C_d, C_H; stagnation C_p = (p - p_inf) / (rho U^2 / 2), C_Q = q / (rho U^3 / 2) from the mean of
        // the stagnation point's two faces; each EMA (alpha = 2/1001) from the first surface sample on
        const double U = K.W_inf[1] / K.W_inf[0];
        const double qd = 0.5 * K.W_inf[0] * (U * U), qh = 0.5 * K.W_inf[0] * ((U * U) * U);
        double v[4] = {sm[0][0] / qd, sm[1][0] / qh, CUDART_NAN, CUDART_NAN};
        if (K.stag0 >= 0) {
            const double* a = d.surf_last + 3 * (size_t)K.stag0;
            const double* b = d.surf_last + 3 * (size_t)K.stag1;
            v[2] = (0.5 * (a[0] + b[0]) - K.W_inf[0] * kR) / qd;
            v[3] = (0.5 * (a[2] + b[2])) / qh;
        }
        const bool first = d.stats[8] == 0;
        for (int q = 0; q < 4; ++q) {
            d.mon[q] = v[q];
            d.mon[4 + q] = first ? v[q] : d.mon[4 + q] + (2.0 / 1001.0) * (v[q] - d.mon[4 + q]);
        }
    }
    // the next step's slots: the particles and holes of this step and the entered ones; after a counting sort
    // the survivors alone, in the other buffer
    // (reserved slots of entered particles count up to the capacity: those past it were not stored)
    const int kept = __ldcg(d.counts + 2);
    if (d.flags[0]) {
        d.counts[0] = kept;
        *d.bufsel = 1 - *d.bufsel;
    } else {
        d.counts[0] = min(__ldcg(d.counts + 4) + __ldcg(d.counts + 7), d.counts[3]);
    }
    // particle-steps of this step: the particles alive at its start, the new ones and those that entered from
    // ghost sources (holes are not particles)
    const unsigned long long alive0 = d.stats[1];
    *dstep += 1;
    d.stats[0] = (unsigned long long)*dstep;
    d.stats[1] = (unsigned long long)kept;
    d.stats[2] = (unsigned long long)d.counts[1];
    d.stats[8] += 1;  // surface samples
    d.stats[9] += alive0 + (unsigned long long)(d.counts[1] + d.counts[6]);
    d.stats[10] += (unsigned long long)d.counts[1];
}
__global__ void __launch_bounds__(kUpdateBlock) k_update(const StepConsts K, Dev d, long long* dstep)
{
    update_body(UGKWP_VB_LAUNCH, K, d, dstep);
}

// ------------------------------------------------------------------ state transfer helpers
template <typename T>
__global__ void k_put_particles(ParticleSoA<T> A, int n, const double* x, const double* y, const double* u,
                                const double* v, const double* w, const double* m, const int* cell,
                                const unsigned long long* pid)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    A.x[i] = T(x[i]); A.y[i] = T(y[i]); A.u[i] = T(u[i]); A.v[i] = T(v[i]); A.w[i] = T(w[i]); A.m[i] = T(m[i]);
    A.cell[i] = cell[i];
    A.pid[i] = pid[i];
}

template <typename T>
__global__ void k_get_particles(ParticleSoA<T> A, int n, double* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = double(A.x[i]); out[n + i] = double(A.y[i]); out[2 * n + i] = double(A.u[i]);
    out[3 * n + i] = double(A.v[i]); out[4 * n + i] = double(A.w[i]); out[5 * n + i] = double(A.m[i]);
}

// after a replacement of the local time steps: 1 / dt_i and the crossing scaling dt_R / dt_L (Eq. 41) of every
// face of every cell, by the same formula as at creation
__global__ void k_set_ratios(Dev d, int C)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    d.rcp[2 * c + 1] = 1.0 / d.dt[c];
    for (int k = 0; k < d.nfc[c]; ++k) {
        const int nb = d.cf64[c].nbr[k];
        const double r = nb >= 0 ? d.dt[nb] / d.dt[c] : 1.0;
        d.cf64[c].ratio[k] = r;
        d.cf32[c].ratio[k] = (float)r;
    }
}

__global__ void k_set_prim(Dev d, int C, const double* prim)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const double rho = prim[4 * c], U = prim[4 * c + 1], V = prim[4 * c + 2], T = prim[4 * c + 3];
    d.W[4 * c] = rho;
    d.W[4 * c + 1] = rho * U;
    d.W[4 * c + 2] = rho * V;
    d.W[4 * c + 3] = rho * (0.5 * (U * U + V * V) + 1.5 * kR * T);
    for (int k = 0; k < 5; ++k) d.wrt[5 * c + k] = 0;
}

__global__ void k_cell_data(const StepConsts K, Dev d, int C, double* out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double* o = out + 8 * c;
    if (K.prec == 0 && !d.wallcell[c] && K.order != 2) {
        // an FP32 cell of the decomposition: its FP32 values (x = dt / tau by the same FP32 division)
        o[0] = d.tau32[c]; o[1] = __fdiv_rn(d.dt32[c], d.tau32[c]); o[2] = d.emx32[c];
    } else {
        o[0] = d.tau[c]; o[1] = d.xr[c]; o[2] = d.emx[c];
    }
    o[3] = (double)d.nhp[c]; o[4] = d.mnew[c];
    o[5] = d.samp[3 * c]; o[6] = d.samp[3 * c + 1]; o[7] = d.samp[3 * c + 2];
}

__global__ void k_wp_field(Dev d, int C, int fx0, int fx1, int fx4, double* out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const long long* r = d.wrt + 5 * c;
    out[4 * c] = ((double)r[0] * pow2(-fx0)) / d.vol[c];
    out[4 * c + 1] = ((double)r[1] * pow2(-fx1)) / d.vol[c];
    out[4 * c + 2] = ((double)r[2] * pow2(-fx1)) / d.vol[c];
    out[4 * c + 3] = ((double)r[4] * pow2(-fx4)) / d.vol[c];
}

// ---------------------------------------------------------------------------- host helpers
int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

ugkwp_status fail(Ctx& c, ugkwp_status st, const char* what)
{
    c.msg = what;
    return st;
}

#define CK(expr)                                                                    \
    do {                                                                            \
        cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ctx.msg = std::string(#expr) + ": " + cudaGetErrorString(e_);           \
            return e_ == cudaErrorMemoryAllocation ? UGKWP_ENOMEM : UGKWP_ECUDA;  \
        }                                                                           \
    } while (0)

// device memory of a context: the caller's allocator when it gave one, else cudaMalloc
cudaError_t raw_alloc(Ctx& ctx, void** q, size_t bytes)
{
    if (ctx.dev_alloc) {
        *q = ctx.dev_alloc(bytes, ctx.stream, ctx.alloc_user);
        return *q ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    return cudaMalloc(q, bytes);
}
void raw_free(Ctx& ctx, void* q)
{
    if (!q) return;
    if (ctx.dev_free) ctx.dev_free(q, ctx.alloc_user);
    else cudaFree(q);
}
// a per-call temporary, returned when it goes out of scope (the calls synchronise their stream before)
struct Tmp {
    Ctx& ctx;
    void* p = nullptr;
    explicit Tmp(Ctx& c) : ctx(c) {}
    ~Tmp()
    {
        if (!p) return;
        cudaStreamSynchronize(ctx.stream);   // nothing queued may still use it (early error returns included)
        raw_free(ctx, p);
    }
    template <typename P> cudaError_t get(P** out, size_t n)
    {
        cudaError_t e = raw_alloc(ctx, &p, (n ? n : 1) * sizeof(P));
        *out = static_cast<P*>(p);
        return e;
    }
};

template <typename P> cudaError_t dalloc(Ctx& ctx, P** p, size_t n)
{
    void* q = nullptr;
    cudaError_t e = raw_alloc(ctx, &q, (n ? n : 1) * sizeof(P));
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(q, 0, (n ? n : 1) * sizeof(P), ctx.stream);
    ctx.allocs.push_back(q);
    *p = static_cast<P*>(q);
    return cudaSuccess;
}

// 64 elements of slack past the capacity: the warp-staged transport kernel copies a tile's last records in
// groups of four (16-byte bulk copies) and may read up to three elements past the particle count
template <typename T> cudaError_t alloc_particles(Ctx& ctx, ParticleSoA<T>& P, size_t cap)
{
    cap += 64;
    cudaError_t e;
    if ((e = dalloc(ctx, &P.x, cap)) || (e = dalloc(ctx, &P.y, cap)) || (e = dalloc(ctx, &P.u, cap)) ||
        (e = dalloc(ctx, &P.v, cap)) || (e = dalloc(ctx, &P.w, cap)) || (e = dalloc(ctx, &P.m, cap)) ||
        (e = dalloc(ctx, &P.cell, cap)) || (e = dalloc(ctx, &P.pid, cap)))
        return e;
    return cudaSuccess;
}

// the warp-staged transport kernels: the stay pass with tile WT = ctx.k.chunk (128 particles per warp tile,
// else 64) and grid_particles / sms CTAs per SM (4, 6 or 8 with 128-particle tiles, 6 or 8 with 64: the
// instantiation compiled for that many resident CTAs), then the flight pass
template <int WT, int MINB> void launch_warp_variant(Ctx& ctx, cudaStream_t s, const PCell<float>& pc)
{
    const StepConsts& K = ctx.k;
    Dev& d = ctx.d;
    k_particles_warp<WT, MINB><<<MINB * ctx.sms, kWWarps * 32, kWWarps * sizeof(WarpSmem<WT>), s>>>(
        K, d, d.pa32, d.pb32, d.cf32, d.dstep);
    k_particles_fly<<<UGKWP_FLY_MINB * ctx.sms, 128, 0, s>>>(K, d, d.pa32, d.pb32, d.cf32, d.dstep);
}
void launch_particles_warp(Ctx& ctx, cudaStream_t s, const PCell<float>& pc)
{
    const int bps = ctx.grid_particles / ctx.sms;
    if (ctx.k.chunk == 128) {
        if (bps >= 7) launch_warp_variant<128, 8>(ctx, s, pc);
        else if (bps >= 5) launch_warp_variant<128, 6>(ctx, s, pc);
        else launch_warp_variant<128, 4>(ctx, s, pc);
    } else {
        if (bps >= 7) launch_warp_variant<64, 8>(ctx, s, pc);
        else launch_warp_variant<64, 6>(ctx, s, pc);
    }
}
template <int WT, int MINB> cudaError_t warp_variant_attr()
{
    return cudaFuncSetAttribute(k_particles_warp<WT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kWWarps * sizeof(WarpSmem<WT>)));
}

}  // namespace

// the per-step kernel sequence (enqueued on s; capturable)
static void enqueue_step(Ctx& ctx, cudaStream_t s, cudaStream_t s2, bool prof)
{
    const StepConsts& K = ctx.k;
    Dev& d = ctx.d;
    const int C = K.C;
    // stage k timed by the event pair (2k, 2k+1) recorded on the stream that runs it
    cudaEvent_t ev[2 * kStages];
    if (prof)
        for (int q = 0; q < 2 * kStages; ++q) cudaEventCreate(&ev[q]);
    auto mark = [&](int q, cudaStream_t st) {
        if (prof) cudaEventRecord(ev[q], st);
    };
    // profiled steps run the second stream's work on the main stream, so that every stage's events time it
    // alone (overlapped, each stage's events would also count the other stream's kernels sharing the SMs)
    cudaStream_t s3 = ctx.stream3;
    if (prof) s2 = s3 = s;
    mark(0, s);
    k_begin_step<<<nblk(2LL * K.F, 256), 256, 0, s>>>(K, d);
    if (K.shakhov) {
        if (K.prec == 0) k_heat_tally<float><<<ctx.grid_particles, 256, 0, s>>>(K, d, d.pa32, d.pb32);
        else k_heat_tally<double><<<ctx.grid_particles, 256, 0, s>>>(K, d, d.pa64, d.pb64);
    }
    k_decompose<<<nblk(C, 128), 128, 0, s>>>(K, d);
    exclusive_scan(d.nhp, d.nhp_off, d.scan_tmp, C, d.counts + 1, s, d.counts, d.err);
    if (K.order == 2) k_gradients<<<nblk(8LL * C, 128), 128, 0, s>>>(K, d);
    mark(1, s);
    // the wave fluxes depend only on the decomposition: they run on a second stream, alongside the
    // particle kernels, and join before the update
    cudaEventRecord(ctx.ev_fork, s);
    cudaStreamWaitEvent(s2, ctx.ev_fork, 0);
    mark(6, s2);
    // ghost particle sources on a third stream: they touch only the slots past the step's particles and the
    // tallies that the transport kernels update atomically, and they join before the sort and the update
    const bool inj = K.n_inj > 0 && !K.wave_only;
    if (inj) {
        if (s3 != s2) cudaStreamWaitEvent(s3, ctx.ev_fork, 0);
        k_inject_params<<<nblk(K.n_inj, 128), 128, 0, s3>>>(K, d);
        if (K.prec == 0) k_inject<float><<<nblk(32LL * K.n_inj, 128), 128, 0, s3>>>(K, d, d.pa32, d.pb32, d.cf32, d.dstep);
        else k_inject<double><<<nblk(32LL * K.n_inj, 128), 128, 0, s3>>>(K, d, d.pa64, d.pb64, d.cf64, d.dstep);
        if (s3 != s) cudaEventRecord(ctx.ev_join3, s3);
    }
    launch_wave_flux(K, d, ctx.sms, s2);
    mark(7, s2);
    cudaEventRecord(ctx.ev_join, s2);
    PCell<float> pc32{d.tau32, d.dt32, d.mnew32, d.samp32, d.hq32, d.emx32};
    PCell<double> pc64{d.tau, d.dt, d.mnew, d.samp, d.hq, d.emx};
    mark(2, s);
    // the particle kernels only where there are particle buffers (not in the particle-free mode)
    const bool parts = !K.wave_only;
    if (parts && K.prec == 0) k_sample<float><<<16 * ctx.sms, 128, 0, s>>>(K, d, d.pa32, d.pb32, pc32, d.dstep);
    else if (parts) k_sample<double><<<16 * ctx.sms, 128, 0, s>>>(K, d, d.pa64, d.pb64, pc64, d.dstep);
    mark(3, s);
    mark(4, s);
    if (parts && K.prec == 0 && ctx.transport == kTransportStaged)
        launch_particles_warp(ctx, s, pc32);
    else if (parts && K.prec == 0)
        k_particles<float><<<ctx.grid_particles, 256, 0, s>>>(K, d, d.pa32, d.pb32, d.cf32, pc32, d.dstep);
    else if (parts)
        k_particles<double><<<ctx.grid_particles, 256, 0, s>>>(K, d, d.pa64, d.pb64, d.cf64, pc64, d.dstep);
    mark(5, s);
    mark(8, s);
    // counting sort every sort_every-th step (kernels return at once on the other steps), after the ghost
    // sources on the second stream have added their survivors
    cudaStreamWaitEvent(s, ctx.ev_join, 0);
    if (inj && s3 != s) cudaStreamWaitEvent(s, ctx.ev_join3, 0);
    exclusive_scan(d.cnt, d.off, d.scan_tmp, C, d.counts + 2, s, nullptr, nullptr, d.flags);
    if (parts && K.prec == 0) k_scatter<float><<<ctx.grid_particles, 256, 0, s>>>(d, d.pa32, d.pb32);
    else if (parts) k_scatter<double><<<ctx.grid_particles, 256, 0, s>>>(d, d.pa64, d.pb64);
    mark(9, s);
    mark(10, s);
    k_update<<<ctx.res_blocks, kUpdateBlock, 0, s>>>(K, d, d.dstep);
    mark(11, s);
    if (prof)
        for (int q = 0; q < 2 * kStages; ++q) ctx.prof_events.push_back(ev[q]);
}

namespace {
// ------------------------------------------------------------- batched persistent step kernel
// One launch advances every case of a batch by one step. The work of a step is a list of items (case, stage,
// blocks b0..b1 of that stage), built on the host in stage-major order: every case's first stage, then every
// case's second stage, and so on, the stages in the order of the step (the algorithm of Sec. III C: decompose,
// sample, transport, then the update; the wave fluxes between decomposition and update). The CTAs of the
// launch take items from a global counter and run each as the blocks of the standalone kernel it stands for
// (same block size, same per-block arithmetic), one block after another. An item waits until every item of
// its case's previous stage has finished; items of other cases do not wait for it, so one case's stage
// boundaries overlap with other cases' work instead of idling the GPU as a grid-wide barrier would.
// No deadlock: an item waits only for items that come earlier in the list, and an item is taken only by a
// running CTA, so the earliest unfinished item can always make progress. Each wait is bounded (a time limit);
// on expiry the CTA raises the batch's abort flag, every CTA stops taking items, and the step reports ELIMIT.
// Scope: production precision, first-order reconstruction and the warp-staged transport with 128-particle
// tiles (the batch falls back to per-case streams for any other case).
enum MkStage : int {
    MS_BEGIN, MS_HEAT, MS_DECOMP, MS_NSCAN_B, MS_NSCAN_T, MS_NSCAN_A, MS_FPREP, MS_FMIX, MS_F32, MS_F64, MS_INJP,
    MS_INJ, MS_SAMPLE, MS_STAY, MS_FLY, MS_CSCAN_B, MS_CSCAN_T, MS_CSCAN_A, MS_SCATTER, MS_UPDATE, MS_COUNT
};
constexpr int kMkThreads = 128;
constexpr int kMkScanTile = 1024;   // elements per scan block (that of exclusive_scan)
constexpr int kMkMaxCases = 64;

struct MkCase {
    StepConsts K;
    Dev d;
    int nv[MS_COUNT];                 // blocks of each stage (0: the stage does not run for this case)
};
// control words of a batch (device): take counter, CTAs finished, abort flag, where a wait ran out, limit
struct MkCtl {
    int next, exited, abort, where;
    unsigned long long limit_ns;
    int stall;                        // test hook: the first wait of the step also waits for a flag nothing sets
    int pad;
};

// exclusive scan of a kMkScanTile-element tile of `in` by 128 threads (eight consecutive elements each); the
// tile's total to tmp[b]. Same outputs as k_scan_blocks (integer sums).
__device__ __forceinline__ void mk_scan_blocks(const VB vb, const int* in, int* out, int* tmp, int n, const int* active)
{
    if (active && !*active) return;
    constexpr int per = kMkScanTile / kMkThreads;
    const int i0 = vb.b * kMkScanTile + threadIdx.x * per;
    int v[per], s = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        v[k] = i0 + k < n ? in[i0 + k] : 0;
        s += v[k];
    }
    int tot;
    int e = block_excl_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < per; ++k) {
        if (i0 + k < n) out[i0 + k] = e;
        e += v[k];
    }
    if (threadIdx.x == 0) tmp[vb.b] = tot;
}
// k_scan_tops by 128 threads (nb <= 1024 block totals, eight per thread)
__device__ __forceinline__ void mk_scan_tops(int* tmp, int nb, int* out, int n, int* total, int* cap, int* err,
                                             const int* active)
{
    if (active && !*active) return;
    constexpr int per = kMkScanTile / kMkThreads;
    const int i0 = threadIdx.x * per;
    int v[per], s = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        v[k] = i0 + k < nb ? tmp[i0 + k] : 0;
        s += v[k];
    }
    int tot;
    int e = block_excl_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < per; ++k) {
        if (i0 + k < nb) tmp[i0 + k] = e;
        e += v[k];
    }
    if (threadIdx.x == 0) {
        out[n] = tot;
        if (cap) {
            if ((long long)cap[0] + tot > (long long)cap[3]) {
                atomicOr(err, ERR_CAPACITY);
                tot = 0;
            }
            cap[4] = cap[0] + tot;
        }
        if (total) *total = tot;
    }
}
__device__ __forceinline__ void mk_scan_add(const VB vb, int* out, const int* tmp, int n, const int* active)
{
    if (active && !*active) return;
    const int add = tmp[vb.b];
    for (int k = threadIdx.x; k < kMkScanTile; k += kMkThreads) {
        const int i = vb.b * kMkScanTile + k;
        if (i < n) out[i] += add;
    }
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// one block b of stage st of a case: the body of the standalone kernel that the stage stands for
__device__ __forceinline__ bool mk_run_block(const MkCase& mc, int st, int b)
{
    const StepConsts& K = mc.K;
    const Dev& d = mc.d;
    const VB vb{b, mc.nv[st]};
    const int nbC = (K.C + kMkScanTile - 1) / kMkScanTile;
    switch (st) {
    case MS_BEGIN: begin_body(vb, K, d); break;
    case MS_HEAT: heat_body<float>(vb, K, d, d.pa32, d.pb32); break;
    case MS_DECOMP: decompose_body(vb, K, d); break;
    case MS_NSCAN_B: mk_scan_blocks(vb, d.nhp, d.nhp_off, d.scan_tmp, K.C, nullptr); break;
    case MS_NSCAN_T: mk_scan_tops(d.scan_tmp, nbC, d.nhp_off, K.C, d.counts + 1, d.counts, d.err, nullptr); break;
    case MS_NSCAN_A: mk_scan_add(vb, d.nhp_off, d.scan_tmp, K.C, nullptr); break;
    case MS_FPREP: wf::flux_prep_body(vb, K, d); break;
    case MS_FMIX: wf::fluxmix_body(vb, K, d); break;
    case MS_F32: wf::flux32_body(vb, K, d); break;
    case MS_F64:
        // the queued faces one per warp (lane 0), as the standalone launch of 32-thread blocks
        wf::flux64_body(K, d, (int)(threadIdx.x & 31), 4 * b + (int)(threadIdx.x >> 5), 4 * vb.n, 1, 0);
        break;
    case MS_INJP: injp_body(vb, K, d); break;
    case MS_INJ: inject_body<float>(vb, K, d, d.pa32, d.pb32, d.cf32, d.dstep); break;
    case MS_SAMPLE: {
        const PCell<float> pc{d.tau32, d.dt32, d.mnew32, d.samp32, d.hq32, d.emx32};
        sample_body<float>(vb, K, d, d.pa32, d.pb32, pc, d.dstep);
        break;
    }
    case MS_STAY: return stay_body<128>(K, d, d.pa32, d.pb32, d.cf32, d.dstep);
    case MS_FLY: fly_body(vb, K, d, d.pa32, d.pb32, d.cf32, d.dstep); break;
    case MS_CSCAN_B: mk_scan_blocks(vb, d.cnt, d.off, d.scan_tmp, K.C, d.flags); break;
    case MS_CSCAN_T: mk_scan_tops(d.scan_tmp, nbC, d.off, K.C, d.counts + 2, nullptr, nullptr, d.flags); break;
    case MS_CSCAN_A: mk_scan_add(vb, d.off, d.scan_tmp, K.C, d.flags); break;
    case MS_SCATTER: scatter_body<float>(vb, d, d.pa32, d.pb32); break;
    case MS_UPDATE: update_body(vb, K, d, d.dstep); break;
    default: break;
    }
    return true;
}

// items: (case, stage, first block, end block); dep[case * MS_COUNT + stage] = (stage waited for, items of it),
// stage -1 for none; done[case * MS_COUNT + stage] counts the finished items of the step
template <int MB>
__global__ void __launch_bounds__(kMkThreads, MB) k_persist_step(const MkCase* __restrict__ cases,
                                                                 const int4* __restrict__ items, int n_items,
                                                                 const int2* __restrict__ dep, int* done, int n_done,
                                                                 MkCtl* ctl, int n_cases)
{
    __shared__ int s_item, s_last;
    for (;;) {
        if (threadIdx.x == 0) {
            int i = ld_relaxed_gpu(&ctl->abort) ? n_items : atomicAdd(&ctl->next, 1);
            if (i < n_items) {
                const int4 it = items[i];
                const int2 dp = dep[it.x * MS_COUNT + it.y];
                // (test hook: with ctl->stall the step's last item waits for one item more than its stage has)
                const int need = dp.y + ((ctl->stall && i == n_items - 1) ? 1 : 0);
                if (dp.x >= 0) {
                    const int* w = done + it.x * MS_COUNT + dp.x;
                    unsigned long long t0 = 0;
                    for (unsigned k = 0;; ++k) {
                        if (ld_acquire_gpu(w) >= need) break;
                        if (ld_relaxed_gpu(&ctl->abort)) { i = n_items; break; }
                        if ((k & 15u) == 15u) {
                            const unsigned long long t = global_ns();
                            if (t0 == 0) {
                                t0 = t;
                            } else if (t - t0 > ctl->limit_ns) {
                                // the wait ran out: stop the batch, record where, flag every case
                                if (atomicCAS(&ctl->abort, 0, 1) == 0) atomicExch(&ctl->where, it.x * MS_COUNT + it.y);
                                for (int q = 0; q < n_cases; ++q) atomicOr(cases[q].d.err, ERR_LIMIT);
                                i = n_items;
                                break;
                            }
                        }
                        __nanosleep(64);
                    }
                    __threadfence();
                }
            }
            s_item = i;
        }
        __syncthreads();
        const int i = s_item;
        if (i >= n_items) break;
        const int4 it = items[i];
        const MkCase& mc = cases[it.x];
        bool ok = true;
        for (int b = it.z; b < it.w && ok; ++b) ok = mk_run_block(mc, it.y, b);
        // a stay-pass tile whose copies did not arrive in time: that warp's shared memory may still be written
        // by them, so this CTA takes no further item and the batch stops
        const bool bad = __syncthreads_or(!ok) != 0;
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + it.x * MS_COUNT + it.y, 1);
            if (bad) {
                if (atomicCAS(&ctl->abort, 0, 1) == 0) atomicExch(&ctl->where, it.x * MS_COUNT + it.y);
                for (int q = 0; q < n_cases; ++q) atomicOr(cases[q].d.err, ERR_LIMIT);
            }
        }
        if (bad) break;
    }
    // the last CTA to finish resets the step's counters for the next launch (the abort flag stays)
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&ctl->exited, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int k = threadIdx.x; k < n_done; k += kMkThreads) done[k] = 0;
        if (threadIdx.x == 0) {
            ctl->next = 0;
            ctl->exited = 0;
        }
    }
}

// blocks of each stage per work item (light per-block work is grouped so that taking an item costs little
// against running it)
constexpr int kMkPer[MS_COUNT] = {4, 1, 2, 2, 1, 4, 4, 1, 1, 1, 4, 2, 1, 1, 1, 2, 1, 4, 1, 2};

// blocks of each stage of one case (np: its particle count when the batch is made, which sizes the stages
// whose blocks walk the particles in grid-stride loops or claim tiles; any count gives the same results)
void mk_plan_case(const Ctx& ctx, int G, long long np, MkCase& mc)
{
    const StepConsts& K = ctx.k;
    const bool parts = !K.wave_only;
    const bool inj = K.n_inj > 0 && parts;
    auto up = [](long long a, long long b) { return (int)((a + b - 1) / b); };
    auto clampG = [&](long long x) { return (int)std::max(1LL, std::min<long long>(G, x)); };
    for (int s = 0; s < MS_COUNT; ++s) mc.nv[s] = 0;
    long long zero = std::max<long long>(2LL * K.F, 3LL * K.nwall);
    if (ctx.d.frec) zero = std::max<long long>(zero, 4LL * K.F);
    if (K.shakhov) zero = std::max<long long>(zero, 9LL * K.C);
    const int nbC = up(K.C, kMkScanTile);
    mc.nv[MS_BEGIN] = clampG(up(zero, 8 * kMkThreads));
    if (K.shakhov) mc.nv[MS_HEAT] = clampG(up(np, 32768));
    mc.nv[MS_DECOMP] = up(K.C, kMkThreads);
    mc.nv[MS_NSCAN_B] = nbC;
    mc.nv[MS_NSCAN_T] = 1;
    mc.nv[MS_NSCAN_A] = nbC;
    mc.nv[MS_FPREP] = up(K.C, kMkThreads);
    if (K.n_mix) mc.nv[MS_FMIX] = up(K.n_mix, kMkThreads);
    mc.nv[MS_F32] = up(K.F, kMkThreads);
    mc.nv[MS_F64] = 4;
    if (inj) {
        mc.nv[MS_INJP] = up(K.n_inj, kMkThreads);
        mc.nv[MS_INJ] = up(32LL * K.n_inj, kMkThreads);
    }
    if (parts) {
        mc.nv[MS_SAMPLE] = clampG(up(K.C, 256));
        mc.nv[MS_STAY] = clampG(up(np, 16384));
        mc.nv[MS_FLY] = clampG(up(np, 65536));
        mc.nv[MS_SCATTER] = clampG(up(np, 16384));
    }
    mc.nv[MS_CSCAN_B] = nbC;
    mc.nv[MS_CSCAN_T] = 1;
    mc.nv[MS_CSCAN_A] = nbC;
    mc.nv[MS_UPDATE] = ctx.res_blocks;
}

template <int MB> cudaError_t mk_occupancy(int* blocks)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_persist_step<MB>, kMkThreads,
                                                         kWWarps * sizeof(WarpSmem<128>));
}
template <int MB>
void mk_launch(int grid, cudaStream_t s, const MkCase* cases, const int4* items, int n_items, const int2* dep,
               int* done, int n_done, MkCtl* ctl, int n_cases)
{
    k_persist_step<MB><<<grid, kMkThreads, kWWarps * sizeof(WarpSmem<128>), s>>>(cases, items, n_items, dep, done,
                                                                               n_done, ctl, n_cases);
}
}  // namespace

}  // namespace ugk

using namespace ugk;

namespace {
ugkwp_status check_device_error(Ctx& ctx)
{
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctx.d.err, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    if (h & ERR_NONPHYS) return fail(ctx, UGKWP_ENONPHYS, "non-physical cell state after the update");
    if (h & ERR_OVERFLOW) return fail(ctx, UGKWP_EOVERFLOW, "fixed-point tally overflow");
    if (h & ERR_CAPACITY) return fail(ctx, UGKWP_ELIMIT, "particle capacity exceeded");
    if (h & ERR_LIMIT) return fail(ctx, UGKWP_ELIMIT, "crossing cap or new-particle cap reached");
    return UGKWP_OK;
}

int ceil_log2(double x)
{
    int e;
    const double m = frexp(x, &e);
    return m == 0.5 ? e - 1 : e;
}

// Connectivity of an unstructured mesh: faces in order of first appearance over the cells and their edges
// (edge k of a cell runs from its vertex k to vertex k + 1), the first cell naming an edge being its L side;
// per cell the local face tables. Validates the mesh (ugkwp_create_unstructured lists the rules).
struct UTopo {
    int C = 0, F = 0;
    std::vector<int> cv, nfc, cface, csgn, cnbr, cnk, cbc;     // per cell (cv, tables: 4 per cell)
    std::vector<int> fa, fb, fl, fr, ftag, fkl, fkr;           // per face
};

bool valid_tag(int t)
{
    return t == UGKWP_BC_WALL || t == UGKWP_BC_FARFIELD || t == UGKWP_BC_FIXED || t == UGKWP_BC_SYMMETRY;
}

ugkwp_status build_topology(const ugkwp_umesh* m, UTopo& t)
{
    const int C = m->n_cells, NV = m->n_vertices;
    t.C = C;
    t.cv.assign(4 * (size_t)C, 0); t.nfc.assign(C, 0);
    t.cface.assign(4 * (size_t)C, 0); t.csgn.assign(4 * (size_t)C, 1); t.cnbr.assign(4 * (size_t)C, -1);
    t.cnk.assign(4 * (size_t)C, 0); t.cbc.assign(4 * (size_t)C, 0);
    std::unordered_map<uint64_t, int> edge;
    edge.reserve(4 * (size_t)C);
    auto key = [NV](int a, int b) { return a < b ? (uint64_t)a * (uint64_t)NV + (uint64_t)b : (uint64_t)b * (uint64_t)NV + (uint64_t)a; };
    for (int c = 0; c < C; ++c) {
        const int32_t* v = m->cells + 4 * (size_t)c;
        const int n = v[3] == -1 ? 3 : 4;
        t.nfc[c] = n;
        for (int q = 0; q < n; ++q) {
            if (v[q] < 0 || v[q] >= NV) return UGKWP_EINVAL;
            for (int r = 0; r < q; ++r)
                if (v[r] == v[q]) return UGKWP_EINVAL;
        }
        for (int q = 0; q < 4; ++q) t.cv[4 * (size_t)c + q] = v[q < n ? q : 2];
        // counter-clockwise and strictly convex: every turn to the left
        for (int q = 0; q < n; ++q) {
            const int a = v[q], b = v[(q + 1) % n], e = v[(q + 2) % n];
            const double ux = m->xv[b] - m->xv[a], uy = m->yv[b] - m->yv[a];
            const double wx = m->xv[e] - m->xv[b], wy = m->yv[e] - m->yv[b];
            if (!(ux * wy - uy * wx > 0.0)) return UGKWP_EINVAL;
        }
        for (int k = 0; k < n; ++k) {
            const int a = v[k], b = v[(k + 1) % n];
            auto it = edge.find(key(a, b));
            int f;
            if (it == edge.end()) {
                f = t.F++;
                edge.emplace(key(a, b), f);
                t.fa.push_back(a); t.fb.push_back(b); t.fl.push_back(c); t.fr.push_back(-1);
                t.ftag.push_back(0); t.fkl.push_back(k); t.fkr.push_back(0);
            } else {
                f = it->second;
                if (t.fr[f] >= 0 || t.fa[f] != b) return UGKWP_EINVAL;   // three cells, or overlapping cells
                t.fr[f] = c;
                t.fkr[f] = k;
            }
            t.cface[4 * (size_t)c + k] = f;
        }
    }
    for (int e = 0; e < m->n_boundary; ++e) {
        const int a = m->boundary[3 * (size_t)e], b = m->boundary[3 * (size_t)e + 1], tag = m->boundary[3 * (size_t)e + 2];
        if (a < 0 || a >= NV || b < 0 || b >= NV || !valid_tag(tag)) return UGKWP_EINVAL;
        auto it = edge.find(key(a, b));
        if (it == edge.end()) return UGKWP_EINVAL;
        const int f = it->second;
        if (t.fr[f] >= 0 || t.ftag[f] != 0) return UGKWP_EINVAL;
        t.ftag[f] = tag;
    }
    for (int f = 0; f < t.F; ++f)
        if (t.fr[f] < 0 && t.ftag[f] == 0) return UGKWP_EINVAL;
    for (int c = 0; c < C; ++c)
        for (int k = 0; k < t.nfc[c]; ++k) {
            const size_t q = 4 * (size_t)c + k;
            const int f = t.cface[q];
            const bool isL = t.fl[f] == c;
            t.csgn[q] = isL ? 1 : -1;
            if (t.fr[f] < 0) { t.cnbr[q] = -1; t.cnk[q] = 0; t.cbc[q] = t.ftag[f]; }
            else { t.cnbr[q] = isL ? t.fr[f] : t.fl[f]; t.cnk[q] = isL ? t.fkr[f] : t.fkl[f]; t.cbc[q] = 0; }
        }
    return UGKWP_OK;
}

ugkwp_status create_impl(const ugkwp_mesh* mesh, const UTopo* topo, const ugkwp_umesh* um, const ugkwp_gas* gas,
                         double Kn, double Ma, double Tw, double cfl, ugkwp_tstep mode, const ugkwp_opts* opts,
                         ugkwp_ctx** out);
}  // namespace

extern "C" {

ugkwp_status ugkwp_create(const ugkwp_mesh* mesh, const ugkwp_gas* gas, double Kn, double Ma, double Tw, double cfl,
                          ugkwp_tstep mode, const ugkwp_opts* opts, ugkwp_ctx** out)
{
    if (!mesh || !gas || !opts || !out || mesh->ni <= 0 || mesh->nj <= 0 || !mesh->xv) return UGKWP_EINVAL;
    if ((long long)mesh->ni * mesh->nj > kMaxCells || opts->n_ref <= 0 || !(cfl > 0.0)) return UGKWP_EINVAL;
    if (mesh->dim != 1 && mesh->dim != 2) return UGKWP_EINVAL;
    if (!(gas->wall_specular >= 0.0 && gas->wall_specular <= 1.0)) return UGKWP_EINVAL;
    if (mesh->dim == 1 && (mesh->nj != 1 || !mesh->bc_imin || !mesh->bc_imax)) return UGKWP_EINVAL;
    if (mesh->dim == 2 && (!mesh->yv || (mesh->periodic_j && mesh->nj < 2))) return UGKWP_EINVAL;
    if (mesh->dim == 1 && ((mesh->bc_imin[0] == UGKWP_BC_PERIODIC) != (mesh->bc_imax[0] == UGKWP_BC_PERIODIC)))
        return UGKWP_EINVAL;
    return create_impl(mesh, nullptr, nullptr, gas, Kn, Ma, Tw, cfl, mode, opts, out);
}

ugkwp_status ugkwp_create_unstructured(const ugkwp_umesh* mesh, const ugkwp_gas* gas, double Kn, double Ma,
                                       double Tw, double cfl, ugkwp_tstep mode, const ugkwp_opts* opts,
                                       ugkwp_ctx** out)
{
    if (!mesh || !gas || !opts || !out || mesh->n_cells <= 0 || mesh->n_vertices <= 0 || !mesh->xv || !mesh->yv ||
        !mesh->cells || mesh->n_boundary < 0 || (mesh->n_boundary > 0 && !mesh->boundary))
        return UGKWP_EINVAL;
    if (mesh->n_cells > kMaxCells || opts->n_ref <= 0 || !(cfl > 0.0)) return UGKWP_EINVAL;
    if (!(gas->wall_specular >= 0.0 && gas->wall_specular <= 1.0)) return UGKWP_EINVAL;
    UTopo topo;
    const ugkwp_status st = build_topology(mesh, topo);
    if (st != UGKWP_OK) return st;
    return create_impl(nullptr, &topo, mesh, gas, Kn, Ma, Tw, cfl, mode, opts, out);
}

}  // extern "C"

namespace {
ugkwp_status create_impl(const ugkwp_mesh* mesh, const UTopo* topo, const ugkwp_umesh* um, const ugkwp_gas* gas,
                         double Kn, double Ma, double Tw, double cfl, ugkwp_tstep mode, const ugkwp_opts* opts,
                         ugkwp_ctx** out)
{
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) return UGKWP_ECUDA;
    ugkwp_ctx* h = new (std::nothrow) ugkwp_ctx;
    if (!h) return UGKWP_ENOMEM;
    Ctx& ctx = h->c;
    *out = nullptr;
    ctx.stream = static_cast<cudaStream_t>(opts->stream);
    if ((opts->dev_alloc == nullptr) != (opts->dev_free == nullptr)) {
        delete h;
        return UGKWP_EINVAL;
    }
    ctx.dev_alloc = opts->dev_alloc;
    ctx.dev_free = opts->dev_free;
    ctx.alloc_user = opts->alloc_user;
    ctx.use_graph = opts->use_graph;
    if (opts->order != 0 && opts->order != 1 && opts->order != 2) {
        delete h;
        return UGKWP_EINVAL;
    }
    if (!(opts->emx_cutoff >= 0.0 && opts->emx_cutoff < 1.0)) {
        delete h;
        return UGKWP_EINVAL;
    }
    if (cudaStreamCreateWithFlags(&ctx.stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx.stream3, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx.ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx.ev_join3, cudaEventDisableTiming) != cudaSuccess) {
        delete h;
        return UGKWP_ECUDA;
    }
    // an unstructured mesh is kept as ni = C, nj = 1 (the structured indices are used only here)
    const int ni = topo ? topo->C : mesh->ni, nj = topo ? 1 : mesh->nj, C = ni * nj;
    const int dim = topo ? 2 : mesh->dim;
    const int periodic_i = !topo && mesh->dim == 1 && mesh->bc_imin[0] == UGKWP_BC_PERIODIC;
    const int F = topo ? topo->F
                       : mesh->dim == 1 ? (periodic_i ? ni : ni + 1) : (ni + 1) * nj + ni * (mesh->periodic_j ? nj : nj + 1);
    ctx.ni = ni; ctx.nj = nj; ctx.periodic_j = topo ? 0 : mesh->periodic_j;
    ctx.Kn = Kn; ctx.Ma = Ma;
    StepConsts& K = ctx.k;
    K.C = C; K.F = F; K.dim = dim; K.n_ref = opts->n_ref; K.wave_only = opts->wave_only;
    K.prec = opts->precision ? 1 : 0;
    K.order = opts->order == 2 ? 2 : 1;
    K.omega = gas->omega; K.Pr = gas->Pr; K.Tw = Tw;
    K.wall_specular = gas->wall_specular;
    K.emx_cutoff = opts->emx_cutoff;
    K.shakhov = gas->Pr != 1.0 && !opts->wave_only;
    K.mu_inf = (15.0 * sqrt(2.0 * 3.14159265358979323846 * 0.5) * Kn) / (2.0 * (5.0 - 2.0 * gas->omega) * (7.0 - 2.0 * gas->omega));
    K.U_inf = Ma * sqrt((5.0 / 3.0) * 0.5 * 1.0);
    K.m2RTw = -2.0 * 0.5 * Tw;
    {
        double Tc = 1.0 + Ma * Ma / 3.0;
        if (Tw > Tc) Tc = Tw;
        if (opts->ghost_state[3] > Tc) Tc = opts->ghost_state[3];
        K.T_cap = 10.0 * Tc;
        double Tm = 1.0;
        if (Tw < Tm) Tm = Tw;
        if (opts->ghost_state[3] > 0.0 && opts->ghost_state[3] < Tm) Tm = opts->ghost_state[3];
        K.T_min = 0.01 * Tm;
        K.U_cap = Ma * sqrt((5.0 / 3.0) * 0.5 * 1.0) + 10.0 * sqrt(0.5 * K.T_cap);
    }
    K.sig_w = sqrt(0.5 * Tw);
    auto cons = [](double rho, double U, double V, double T, double* W) {
        W[0] = rho; W[1] = rho * U; W[2] = rho * V; W[3] = rho * (0.5 * (U * U + V * V) + 1.5 * 0.5 * T);
    };
    cons(1.0, K.U_inf, 0.0, 1.0, K.W_inf);
    cons(opts->ghost_state[0], opts->ghost_state[1], opts->ghost_state[2], opts->ghost_state[3], K.W_fix);
    K.k0 = (uint32_t)opts->seed ^ opts->case_id;
    K.k1 = (uint32_t)(opts->seed >> 32);
    ctx.capacity = opts->capacity > 0 ? opts->capacity : (int)std::min<long long>(4LL * opts->n_ref * C, 0x7fffffffLL - 64);
    ugkwp_status st = UGKWP_OK;
    auto build = [&]() -> ugkwp_status {
        Dev& d = ctx.d;
        // host mesh -> device
        const int nv = topo ? um->n_vertices : mesh->dim == 1 ? ni + 1 : (ni + 1) * (nj + 1);
        double *xv, *yv;
        CK(dalloc(ctx, &xv, nv)); CK(dalloc(ctx, &yv, nv));
        CK(cudaMemcpyAsync(xv, topo ? um->xv : mesh->xv, sizeof(double) * nv, cudaMemcpyHostToDevice, ctx.stream));
        if (dim == 2)
            CK(cudaMemcpyAsync(yv, topo ? um->yv : mesh->yv, sizeof(double) * nv, cudaMemcpyHostToDevice, ctx.stream));
        MeshDev m{ni, nj, dim, ctx.periodic_j, periodic_i, F, xv, yv, nullptr, nullptr, nullptr, nullptr};
        if (!topo) {
            int *bci, *bco, *bcjl, *bcjh;
            CK(dalloc(ctx, &bci, nj)); CK(dalloc(ctx, &bco, nj)); CK(dalloc(ctx, &bcjl, ni)); CK(dalloc(ctx, &bcjh, ni));
            CK(cudaMemcpyAsync(bci, mesh->bc_imin, sizeof(int) * nj, cudaMemcpyHostToDevice, ctx.stream));
            CK(cudaMemcpyAsync(bco, mesh->bc_imax, sizeof(int) * nj, cudaMemcpyHostToDevice, ctx.stream));
            if (mesh->dim == 2 && !mesh->periodic_j) {
                if (!mesh->bc_jmin || !mesh->bc_jmax) return fail(ctx, UGKWP_EINVAL, "missing j boundary tags");
                CK(cudaMemcpyAsync(bcjl, mesh->bc_jmin, sizeof(int) * ni, cudaMemcpyHostToDevice, ctx.stream));
                CK(cudaMemcpyAsync(bcjh, mesh->bc_jmax, sizeof(int) * ni, cudaMemcpyHostToDevice, ctx.stream));
            }
            m.bc_imin = bci; m.bc_imax = bco; m.bc_jmin = bcjl; m.bc_jmax = bcjh;
        }
        CK(dalloc(ctx, &d.vol, C)); CK(dalloc(ctx, &d.rcp, 2 * C)); CK(dalloc(ctx, &d.wallcell, C)); CK(dalloc(ctx, &d.xc, C)); CK(dalloc(ctx, &d.yc, C)); CK(dalloc(ctx, &d.dt, C));
        CK(dalloc(ctx, &d.nfc, C)); CK(dalloc(ctx, &d.cf32, C)); CK(dalloc(ctx, &d.cf64, C));
        CK(dalloc(ctx, &d.cshift, 4 * C)); CK(dalloc(ctx, &d.cvx, 4 * C)); CK(dalloc(ctx, &d.cvy, 4 * C));
        CK(dalloc(ctx, &d.fL, F)); CK(dalloc(ctx, &d.fR, F)); CK(dalloc(ctx, &d.fbc, F)); CK(dalloc(ctx, &d.fwall, F));
        CK(dalloc(ctx, &d.fnx, F)); CK(dalloc(ctx, &d.fny, F)); CK(dalloc(ctx, &d.fs, F));
        CK(dalloc(ctx, &d.fdL, F)); CK(dalloc(ctx, &d.fdR, F)); CK(dalloc(ctx, &d.face_f64, F));
        CK(dalloc(ctx, &d.fax, F)); CK(dalloc(ctx, &d.fay, F)); CK(dalloc(ctx, &d.fex, F)); CK(dalloc(ctx, &d.fey, F));
        double *fd, *cnx, *cny, *cd, *dtpart;
        int *cface, *csgn, *cnbr, *cnk, *cbc, *flag, *widx;
        CK(dalloc(ctx, &fd, F)); CK(dalloc(ctx, &cnx, 4 * C)); CK(dalloc(ctx, &cny, 4 * C)); CK(dalloc(ctx, &cd, 4 * C));
        CK(dalloc(ctx, &cface, 4 * C)); CK(dalloc(ctx, &csgn, 4 * C)); CK(dalloc(ctx, &cnbr, 4 * C));
        CK(dalloc(ctx, &cnk, 4 * C)); CK(dalloc(ctx, &cbc, 4 * C)); CK(dalloc(ctx, &flag, F)); CK(dalloc(ctx, &widx, F + 1));
        const int nbdt = nblk(C, 256);
        CK(dalloc(ctx, &dtpart, nbdt));
        CK(dalloc(ctx, &d.scan_tmp, kScanBlock));
        if (topo) {
            int *cv, *fa, *fb, *fl, *fr, *ftag;
            CK(dalloc(ctx, &cv, 4 * C)); CK(dalloc(ctx, &fa, F)); CK(dalloc(ctx, &fb, F)); CK(dalloc(ctx, &fl, F));
            CK(dalloc(ctx, &fr, F)); CK(dalloc(ctx, &ftag, F));
            auto up = [&](int* dst, const std::vector<int>& src) {
                return cudaMemcpyAsync(dst, src.data(), sizeof(int) * src.size(), cudaMemcpyHostToDevice, ctx.stream);
            };
            CK(up(cv, topo->cv)); CK(up(fa, topo->fa)); CK(up(fb, topo->fb)); CK(up(fl, topo->fl));
            CK(up(fr, topo->fr)); CK(up(ftag, topo->ftag));
            CK(up(d.nfc, topo->nfc)); CK(up(cface, topo->cface)); CK(up(csgn, topo->csgn)); CK(up(cnbr, topo->cnbr));
            CK(up(cnk, topo->cnk)); CK(up(cbc, topo->cbc));
            const UMeshDev um_d{C, F, xv, yv, cv, fa, fb, fl, fr, ftag};
            k_setup_faces_u<<<nblk(F, 128), 128, 0, ctx.stream>>>(um_d, d, fd);
            k_setup_cells_u<<<nblk(C, 128), 128, 0, ctx.stream>>>(um_d, d, fd, cface, csgn, cnx, cny, cd);
        } else {
            k_setup_faces<<<nblk(F, 128), 128, 0, ctx.stream>>>(m, d, fd);
            k_setup_cells<<<nblk(C, 128), 128, 0, ctx.stream>>>(m, d, fd, cface, csgn, cnbr, cnk, cbc, cnx, cny, cd);
        }
        k_setup_face_dist<<<nblk(F, 128), 128, 0, ctx.stream>>>(m, d, fd);
        const double cs = K.U_inf + 3.0 * sqrt(0.5 * 1.0);
        k_setup_dt<<<nbdt, 256, 0, ctx.stream>>>(d, C, cface, cfl, cs, dtpart);
        if (mode == UGKWP_GTS) k_setup_gts<<<nblk(C, 256), 256, 0, ctx.stream>>>(d, C, dtpart, nbdt);
        k_setup_tables<<<nblk(C, 128), 128, 0, ctx.stream>>>(d, C, cface, csgn, cnbr, cnk, cbc, cnx, cny, cd, K.prec == 0);
        k_wall_flags<<<nblk(F, 128), 128, 0, ctx.stream>>>(d, F, flag);
        int* nwall_d;
        CK(dalloc(ctx, &nwall_d, 1));
        exclusive_scan(flag, widx, d.scan_tmp, F, nwall_d, ctx.stream);
        int nwall = 0;
        CK(cudaMemcpyAsync(&nwall, nwall_d, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaStreamSynchronize(ctx.stream));
        K.nwall = nwall;
        CK(dalloc(ctx, &d.wall_face, nwall));
        k_wall_index<<<nblk(F, 128), 128, 0, ctx.stream>>>(d, F, widx);
        {
            // the stagnation point of the monitors: the two wall faces whose fluid-cell normals face the
            // freestream (+x) most, ties to the lower index, if the best is within 60 degrees of it
            std::vector<int> wf(std::max(nwall, 1));
            std::vector<double> fnx(F);
            CK(cudaMemcpyAsync(wf.data(), d.wall_face, sizeof(int) * nwall, cudaMemcpyDeviceToHost, ctx.stream));
            CK(cudaMemcpyAsync(fnx.data(), d.fnx, sizeof(double) * F, cudaMemcpyDeviceToHost, ctx.stream));
            CK(cudaStreamSynchronize(ctx.stream));
            int a = -1, b = -1;
            for (int iw = 0; iw < nwall; ++iw) {
                const double nx = fnx[wf[iw]];
                if (a < 0 || nx > fnx[wf[a]]) { b = a; a = iw; }
                else if (b < 0 || nx > fnx[wf[b]]) b = iw;
            }
            K.stag0 = K.stag1 = -1;
            if (a >= 0 && b >= 0 && fnx[wf[a]] > 0.5) {
                K.stag0 = std::min(a, b);
                K.stag1 = std::max(a, b);
            }
        }
        {
            // far-field and fixed faces in face order: ghost particle sources, with the face's local index in
            // its fluid cell
            std::vector<int> fbc(F), fl(F), cfh(4 * (size_t)C), nfc(C);
            CK(cudaMemcpyAsync(fbc.data(), d.fbc, sizeof(int) * F, cudaMemcpyDeviceToHost, ctx.stream));
            CK(cudaMemcpyAsync(fl.data(), d.fL, sizeof(int) * F, cudaMemcpyDeviceToHost, ctx.stream));
            CK(cudaMemcpyAsync(cfh.data(), cface, sizeof(int) * 4 * (size_t)C, cudaMemcpyDeviceToHost, ctx.stream));
            CK(cudaMemcpyAsync(nfc.data(), d.nfc, sizeof(int) * C, cudaMemcpyDeviceToHost, ctx.stream));
            CK(cudaStreamSynchronize(ctx.stream));
            std::vector<int> jf, jk;
            for (int f = 0; f < F; ++f) {
                if (fbc[f] != UGKWP_BC_FARFIELD && fbc[f] != UGKWP_BC_FIXED) continue;
                const int L = fl[f];
                int kk = -1;
                for (int k = 0; k < nfc[L]; ++k) if (cfh[4 * (size_t)L + k] == f) kk = k;
                jf.push_back(f);
                jk.push_back(kk);
            }
            K.n_inj = (int)jf.size();
            const int n1 = std::max(K.n_inj, 1);
            CK(dalloc(ctx, &d.inj_face, n1)); CK(dalloc(ctx, &d.inj_k, n1)); CK(dalloc(ctx, &d.inj_n, n1));
            CK(dalloc(ctx, &d.inj_par, 5 * n1));
            if (K.n_inj) {
                CK(cudaMemcpyAsync(d.inj_face, jf.data(), sizeof(int) * K.n_inj, cudaMemcpyHostToDevice, ctx.stream));
                CK(cudaMemcpyAsync(d.inj_k, jk.data(), sizeof(int) * K.n_inj, cudaMemcpyHostToDevice, ctx.stream));
            }
            CK(cudaStreamSynchronize(ctx.stream));
        }
        // fixed-point exponents: per-cell sums stay below 2^61 for up to 1024 x freestream density in the
        // largest cell and speeds up to U_inf + 10 sqrt(R T_max)
        std::vector<double> vol(C);
        CK(cudaMemcpyAsync(vol.data(), d.vol, sizeof(double) * C, cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaStreamSynchronize(ctx.stream));
        double vmax = 0.0, area = 0.0;
        for (int c = 0; c < C; ++c) {
            if (!(vol[c] > 0.0)) return fail(ctx, UGKWP_EINVAL, "cell with non-positive area");
            if (vol[c] > vmax) vmax = vol[c];
            area += vol[c];
        }
        // residual normalisation (ugkwp_residual): S_c sqrt(sum_i Omega_i) / L_ref, L_ref = 1,
        // S = (rho c, rho c^2, rho c^2, rho c^3 / 2), rho_inf = 1, c = U_inf + sqrt(gamma R T_inf)
        {
            const double cs = K.U_inf + sqrt((5.0 / 3.0) * 0.5 * 1.0), ra = sqrt(area);
            ctx.res_scale[0] = cs * ra;
            ctx.res_scale[1] = (cs * cs) * ra;
            ctx.res_scale[2] = ctx.res_scale[1];
            ctx.res_scale[3] = (0.5 * ((cs * cs) * cs)) * ra;
        }
        double Tmax = 1.0;
        if (Tw > Tmax) Tmax = Tw;
        if (opts->ghost_state[3] > Tmax) Tmax = opts->ghost_state[3];
        const double speed = K.U_inf + 10.0 * sqrt(0.5 * Tmax);
        const double b0 = 1024.0 * vmax;
        K.fx0 = 61 - ceil_log2(b0);
        K.fx1 = 61 - ceil_log2(b0 * speed);
        K.fx4 = 61 - ceil_log2(b0 * (0.5 * (speed * speed)));
        K.fx_s2 = 61 - ceil_log2(b0 * (speed * speed));
        K.fx_s3 = 61 - ceil_log2(b0 * (speed * speed * speed));
        {
            double tab[6][kSeries];
            double f1 = 1.0;   // (k+1)!
            for (int k = 0; k < kSeries; ++k) {
                if (k > 0) f1 *= (double)(k + 1);
                const double f2 = f1 * (double)(k + 2), f3 = f2 * (double)(k + 3);
                tab[0][k] = 1.0 / f1;
                tab[1][k] = 1.0 / f2;
                tab[2][k] = 1.0 / f3;
                tab[3][k] = (double)(k + 1) / f2;
                tab[4][k] = (double)(k + 1) / f3;
                tab[5][k] = (double)((k + 1) * (k + 2)) / (2.0 * f3);
            }
            CK(cudaMemcpyToSymbol(c_series, tab, sizeof tab));
            float tab32[6][kSeries32];
            for (int q = 0; q < 6; ++q)
                for (int k = 0; k < kSeries32; ++k) tab32[q][k] = (float)tab[q][k];
            CK(cudaMemcpyToSymbol(c_series32, tab32, sizeof tab32));
            double tf[5][kSeries];
            for (int k = 0; k < kSeries; ++k) {
                tf[0][k] = tab[0][k]; tf[1][k] = tab[1][k]; tf[2][k] = tab[2][k]; tf[3][k] = tab[4][k]; tf[4][k] = tab[3][k];
            }
            CK(flux_set_tables(&tf[0][0], ctx.stream));
            CK(cudaStreamSynchronize(ctx.stream));
        }
        // state and per-step arrays
        CK(dalloc(ctx, &d.W, 4 * C)); CK(dalloc(ctx, &d.wrt, 5 * C)); CK(dalloc(ctx, &d.wprev, 5 * C));
        CK(dalloc(ctx, &d.wm, 5 * C)); CK(dalloc(ctx, &d.wpl, 5 * C)); CK(dalloc(ctx, &d.wcol, 5 * C)); CK(dalloc(ctx, &d.cross, 2 * F));
        CK(dalloc(ctx, &d.wallt, 3 * std::max(nwall, 1)));
        CK(dalloc(ctx, &d.tau, C)); CK(dalloc(ctx, &d.xr, C)); CK(dalloc(ctx, &d.emx, C)); CK(dalloc(ctx, &d.Wh, 4 * C));
        CK(dalloc(ctx, &d.co, 7 * C)); CK(dalloc(ctx, &d.mnew, C)); CK(dalloc(ctx, &d.samp, 3 * C));
        CK(dalloc(ctx, &d.whq, 9 * C)); CK(dalloc(ctx, &d.hq, 3 * C)); CK(dalloc(ctx, &d.hq32, 3 * C));
        CK(dalloc(ctx, &d.nhp, C)); CK(dalloc(ctx, &d.nhp_off, C + 1));
        CK(dalloc(ctx, &d.scells, C)); CK(dalloc(ctx, &d.nscell, 1));
        CK(dalloc(ctx, &d.cnt, C)); CK(dalloc(ctx, &d.off, C + 1)); CK(dalloc(ctx, &d.cur, C));
        CK(dalloc(ctx, &d.flux, 4 * F));
        ctx.res_blocks = nblk((long long)C + nwall, kUpdateBlock);
        CK(dalloc(ctx, &d.res_part, 4 * ctx.res_blocks)); CK(dalloc(ctx, &d.res, 8));
        CK(dalloc(ctx, &d.mon, 8));
        {
            const double nan8[8] = {NAN, NAN, NAN, NAN, NAN, NAN, NAN, NAN};
            CK(cudaMemcpyAsync(d.mon, nan8, sizeof nan8, cudaMemcpyHostToDevice, ctx.stream));
            CK(cudaStreamSynchronize(ctx.stream));
        }
        CK(dalloc(ctx, &d.chi_ema, C));
        CK(dalloc(ctx, &d.surf_sum, 3 * std::max(nwall, 1))); CK(dalloc(ctx, &d.surf_last, 3 * std::max(nwall, 1)));
        CK(dalloc(ctx, &d.counts, 8)); CK(dalloc(ctx, &d.stats, 16)); CK(dalloc(ctx, &d.err, 1));
        CK(dalloc(ctx, &d.bufsel, 1)); CK(dalloc(ctx, &d.flags, 4)); CK(dalloc(ctx, &d.nretry, 1));
        CK(dalloc(ctx, &d.retry, F)); CK(dalloc(ctx, &d.done, 1));
        {
            // faces evaluated wholly in FP64: all in the FP64 mode, none in production mode (there the faces of
            // wall cells, flagged in face_f64, weight FP32 moments with FP64 time integrals)
            std::vector<int> ff(F), fb(F);
            CK(cudaMemcpyAsync(ff.data(), d.face_f64, sizeof(int) * F, cudaMemcpyDeviceToHost, ctx.stream));
            CK(cudaMemcpyAsync(fb.data(), d.fR, sizeof(int) * F, cudaMemcpyDeviceToHost, ctx.stream));
            CK(cudaStreamSynchronize(ctx.stream));
            std::vector<int> list, mix;
            for (int f = 0; f < F; ++f) {
                if (K.prec == 1) ff[f] = 1;
                if (K.prec == 1) list.push_back(f);
                else if (ff[f]) mix.push_back(f);
            }
            K.n_f64 = (int)list.size();
            K.n_mix = (int)mix.size();
            CK(dalloc(ctx, &d.f64list, std::max(K.n_f64, 1)));
            CK(dalloc(ctx, &d.mixlist, std::max(K.n_mix, 1)));
            if (K.n_mix)
                CK(cudaMemcpyAsync(d.mixlist, mix.data(), sizeof(int) * K.n_mix, cudaMemcpyHostToDevice, ctx.stream));
            CK(cudaMemcpyAsync(d.face_f64, ff.data(), sizeof(int) * F, cudaMemcpyHostToDevice, ctx.stream));
            if (K.n_f64)
                CK(cudaMemcpyAsync(d.f64list, list.data(), sizeof(int) * K.n_f64, cudaMemcpyHostToDevice, ctx.stream));
            CK(cudaStreamSynchronize(ctx.stream));
        }
        K.sort_every = UGKWP_SORT_EVERY;
        K.chunk = UGKWP_CHUNK;
        CK(dalloc(ctx, &d.tau32, C)); CK(dalloc(ctx, &d.dt32, C)); CK(dalloc(ctx, &d.mnew32, C));
        CK(dalloc(ctx, &d.emx32, C)); CK(dalloc(ctx, &d.cst32, C));
        if (K.prec == 0) {
            CK(dalloc(ctx, &d.w32, C)); CK(dalloc(ctx, &d.wh32, C)); CK(dalloc(ctx, &d.dp32, C));
            CK(dalloc(ctx, &d.co32, 8 * (size_t)C));
        }
        if (opts->record_faces && !K.wave_only) CK(dalloc(ctx, &d.frec, 4 * (size_t)F));
        if (K.order == 2) CK(dalloc(ctx, &d.grad, 16 * (size_t)C));
        CK(dalloc(ctx, &d.samp32, 3 * C));
        CK(dalloc(ctx, &d.dstep, 1));
        int sms = 148;
        int dev = 0;
        CK(cudaGetDevice(&dev));
        ctx.device = dev;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        ctx.grid_particles = sms * 4;
        ctx.sms = sms;
        ctx.transport = K.prec == 0 ? kTransportStaged : kTransportWarp;
        if (K.prec == 0) {
            ctx.k.chunk = 128;
            ctx.grid_particles = sms * 8;
            CK((warp_variant_attr<64, 6>()));
            CK((warp_variant_attr<64, 8>()));
            CK((warp_variant_attr<128, 4>()));
            CK((warp_variant_attr<128, 6>()));
            CK((warp_variant_attr<128, 8>()));
        }
        if (!K.wave_only) {
            if (K.prec == 0) {
                CK(alloc_particles(ctx, d.pa32, ctx.capacity)); CK(alloc_particles(ctx, d.pb32, ctx.capacity));
                CK(dalloc(ctx, &d.xq_i, (size_t)ctx.capacity)); CK(dalloc(ctx, &d.xq_t, (size_t)ctx.capacity));
                CK(dalloc(ctx, &d.xq.x, (size_t)ctx.capacity)); CK(dalloc(ctx, &d.xq.y, (size_t)ctx.capacity));
                CK(dalloc(ctx, &d.xq.u, (size_t)ctx.capacity)); CK(dalloc(ctx, &d.xq.v, (size_t)ctx.capacity));
                CK(dalloc(ctx, &d.xq.cell, (size_t)ctx.capacity)); CK(dalloc(ctx, &d.xq.pid, (size_t)ctx.capacity));
                CK(dalloc(ctx, &d.nxq, 1));
            }
            else { CK(alloc_particles(ctx, d.pa64, ctx.capacity)); CK(alloc_particles(ctx, d.pb64, ctx.capacity)); }
        }
        const int cnt_init[8] = {0, 0, 0, K.wave_only ? 0 : ctx.capacity, 0, 0, 0, 0};
        CK(cudaMemcpyAsync(d.counts, cnt_init, sizeof cnt_init, cudaMemcpyHostToDevice, ctx.stream));
        // freestream initial state
        std::vector<double> prim(4 * (size_t)C);
        for (int c = 0; c < C; ++c) { prim[4 * c] = 1.0; prim[4 * c + 1] = K.U_inf; prim[4 * c + 2] = 0.0; prim[4 * c + 3] = 1.0; }
        double* dprim;
        CK(dalloc(ctx, &dprim, 4 * C));
        CK(cudaMemcpyAsync(dprim, prim.data(), sizeof(double) * 4 * C, cudaMemcpyHostToDevice, ctx.stream));
        k_set_prim<<<nblk(C, 128), 128, 0, ctx.stream>>>(d, C, dprim);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(ctx.stream));
        return UGKWP_OK;
    };
    st = build();
    if (st != UGKWP_OK) {
        *out = h;   // let the caller read the message, then destroy
        return st;
    }
    *out = h;
    return UGKWP_OK;
}
}  // namespace

extern "C" {

void ugkwp_destroy(ugkwp_ctx* h)
{
    if (!h) return;
    Ctx& ctx = h->c;
    if (ctx.stream) cudaStreamSynchronize(ctx.stream);
    else cudaDeviceSynchronize();
    if (ctx.graph) cudaGraphExecDestroy(ctx.graph);
    for (cudaEvent_t e : ctx.prof_events) cudaEventDestroy(e);
    if (ctx.stream2) cudaStreamSynchronize(ctx.stream2);
    if (ctx.stream3) cudaStreamSynchronize(ctx.stream3);
    for (void* p : ctx.allocs) raw_free(ctx, p);
    if (ctx.stream2) cudaStreamDestroy(ctx.stream2);
    if (ctx.stream3) cudaStreamDestroy(ctx.stream3);
    if (ctx.ev_fork) cudaEventDestroy(ctx.ev_fork);
    if (ctx.ev_join) cudaEventDestroy(ctx.ev_join);
    if (ctx.ev_join3) cudaEventDestroy(ctx.ev_join3);
    delete h;
}

ugkwp_status ugkwp_step(ugkwp_ctx* h, int32_t n)
{
    if (!h || n < 0) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    if (ctx.use_graph && !ctx.profiling) {
        if (!ctx.graph) {
            cudaStream_t cap;
            CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            enqueue_step(ctx, cap, ctx.stream2, false);
            CK(cudaStreamEndCapture(cap, &g));
            CK(cudaGraphInstantiate(&ctx.graph, g, 0));
            cudaGraphDestroy(g);
            cudaStreamDestroy(cap);
        }
        for (int32_t s = 0; s < n; ++s) CK(cudaGraphLaunch(ctx.graph, ctx.stream));
    } else {
        for (int32_t s = 0; s < n; ++s) enqueue_step(ctx, ctx.stream, ctx.stream2, ctx.profiling != 0);
    }
    CK(cudaGetLastError());
    ctx.step += n;
    return UGKWP_OK;
}

ugkwp_status ugkwp_residual(ugkwp_ctx* h, double* out)
{
    if (!h || !out) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    double r[8];
    CK(cudaMemcpyAsync(r, ctx.d.res, sizeof r, cudaMemcpyDeviceToHost, ctx.stream));
    ugkwp_status st = check_device_error(ctx);
    for (int q = 0; q < 4; ++q) { out[q] = r[q] / ctx.res_scale[q]; out[4 + q] = r[q]; }
    return st;
}

ugkwp_status ugkwp_surface(ugkwp_ctx* h, double* p, double* tau, double* q, int32_t n_wall, int32_t averaged)
{
    if (!h || !p || !tau || !q) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    if (n_wall != ctx.k.nwall) return fail(ctx, UGKWP_EINVAL, "n_wall does not match the mesh");
    std::vector<double> s(3 * (size_t)std::max(n_wall, 1));
    unsigned long long st_h[16];
    CK(cudaMemcpyAsync(s.data(), averaged ? ctx.d.surf_sum : ctx.d.surf_last, sizeof(double) * 3 * n_wall,
                       cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaMemcpyAsync(st_h, ctx.d.stats, sizeof st_h, cudaMemcpyDeviceToHost, ctx.stream));
    ugkwp_status st = check_device_error(ctx);
    const double dv = averaged && st_h[8] > 0 ? (double)st_h[8] : 1.0;
    for (int i = 0; i < n_wall; ++i) { p[i] = s[3 * i] / dv; tau[i] = s[3 * i + 1] / dv; q[i] = s[3 * i + 2] / dv; }
    return st;
}

ugkwp_status ugkwp_monitors(ugkwp_ctx* h, double* out)
{
    if (!h || !out) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    CK(cudaMemcpyAsync(out, ctx.d.mon, sizeof(double) * 8, cudaMemcpyDeviceToHost, ctx.stream));
    return check_device_error(ctx);
}

ugkwp_status ugkwp_reset_surface(ugkwp_ctx* h)
{
    if (!h) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    CK(cudaMemsetAsync(ctx.d.surf_sum, 0, sizeof(double) * 3 * std::max(ctx.k.nwall, 1), ctx.stream));
    CK(cudaMemsetAsync(ctx.d.stats + 8, 0, sizeof(unsigned long long), ctx.stream));
    return UGKWP_OK;
}

ugkwp_status ugkwp_set_field(ugkwp_ctx* h, const double* prim)
{
    if (!h || !prim) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    const int C = ctx.k.C;
    for (int c = 0; c < C; ++c)
        if (!(prim[4 * c] > 0.0) || !(prim[4 * c + 3] > 0.0)) return fail(ctx, UGKWP_EINVAL, "non-positive density or temperature");
    double* dp = nullptr;
    Tmp t(ctx);
    CK(t.get(&dp, 4 * (size_t)C));
    CK(cudaMemcpyAsync(dp, prim, sizeof(double) * 4 * C, cudaMemcpyHostToDevice, ctx.stream));
    k_set_prim<<<nblk(C, 128), 128, 0, ctx.stream>>>(ctx.d, C, dp);
    int zero = 0;
    CK(cudaMemcpyAsync(ctx.d.counts, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    return UGKWP_OK;
}

ugkwp_status ugkwp_set_time_steps(ugkwp_ctx* h, const double* dt)
{
    if (!h || !dt) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    const int C = ctx.k.C;
    for (int c = 0; c < C; ++c)
        if (!(dt[c] > 0.0) || !std::isfinite(dt[c])) return fail(ctx, UGKWP_EINVAL, "time steps must be finite and positive");
    CK(cudaMemcpyAsync(ctx.d.dt, dt, sizeof(double) * C, cudaMemcpyHostToDevice, ctx.stream));
    k_set_ratios<<<nblk(C, 128), 128, 0, ctx.stream>>>(ctx.d, C);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx.stream));
    return UGKWP_OK;
}

ugkwp_status ugkwp_get_field(ugkwp_ctx* h, double* W, double* Wp)
{
    if (!h || !W) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    const int C = ctx.k.C;
    CK(cudaMemcpyAsync(W, ctx.d.W, sizeof(double) * 4 * C, cudaMemcpyDeviceToHost, ctx.stream));
    if (Wp) {
        double* dp = nullptr;
        Tmp t(ctx);
        CK(t.get(&dp, 4 * (size_t)C));
        k_wp_field<<<nblk(C, 128), 128, 0, ctx.stream>>>(ctx.d, C, ctx.k.fx0, ctx.k.fx1, ctx.k.fx4, dp);
        CK(cudaMemcpyAsync(Wp, dp, sizeof(double) * 4 * C, cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaStreamSynchronize(ctx.stream));
    }
    return check_device_error(ctx);
}

ugkwp_status ugkwp_stats(ugkwp_ctx* h, int64_t* out)
{
    if (!h || !out) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    unsigned long long s[16];
    CK(cudaMemcpyAsync(s, ctx.d.stats, sizeof s, cudaMemcpyDeviceToHost, ctx.stream));
    ugkwp_status st = check_device_error(ctx);
    for (int k = 0; k < 8; ++k) out[k] = (int64_t)s[k];
    out[8] = (int64_t)s[9];
    out[9] = (int64_t)s[10];
    out[10] = (int64_t)s[11];
    out[11] = (int64_t)s[12];
    out[12] = (int64_t)s[13];
    return st;
}

// particles alive (the slots of the particle buffer also hold holes between counting sorts)
int64_t ugkwp_num_particles(ugkwp_ctx* h)
{
    if (!h) return -1;
    Ctx& ctx = h->c;
    unsigned long long n = 0;
    if (cudaMemcpyAsync(&n, ctx.d.stats + 1, sizeof n, cudaMemcpyDeviceToHost, ctx.stream) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(ctx.stream) != cudaSuccess) return -1;
    return (int64_t)n;
}

ugkwp_status ugkwp_get_particles(ugkwp_ctx* h, int64_t cap, uint64_t* pid, int32_t* cell, double* x, double* y,
                                 double* u, double* v, double* w, double* m)
{
    if (!h) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    const int64_t n = ugkwp_num_particles(h);
    if (n < 0) return fail(ctx, UGKWP_ECUDA, "reading the particle count");
    if (cap < n) return fail(ctx, UGKWP_EINVAL, "host arrays too short");
    if (n == 0) return UGKWP_OK;
    int slots = 0, sel = 0;
    CK(cudaMemcpyAsync(&slots, ctx.d.counts, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaMemcpyAsync(&sel, ctx.d.bufsel, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    // every slot to the host, then the particles (cell >= 0) in slot order
    const size_t ns = (size_t)slots;
    std::vector<double> hv(6 * ns);
    std::vector<uint64_t> hp(ns);
    std::vector<int32_t> hc(ns);
    double* tmp = nullptr;
    Tmp t(ctx);
    CK(t.get(&tmp, 6 * ns));
    if (ctx.k.prec == 0) {
        const ParticleSoA<float>& A = sel ? ctx.d.pb32 : ctx.d.pa32;
        k_get_particles<float><<<nblk(slots, 256), 256, 0, ctx.stream>>>(A, slots, tmp);
        CK(cudaMemcpyAsync(hp.data(), A.pid, sizeof(uint64_t) * ns, cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaMemcpyAsync(hc.data(), A.cell, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, ctx.stream));
    } else {
        const ParticleSoA<double>& A = sel ? ctx.d.pb64 : ctx.d.pa64;
        k_get_particles<double><<<nblk(slots, 256), 256, 0, ctx.stream>>>(A, slots, tmp);
        CK(cudaMemcpyAsync(hp.data(), A.pid, sizeof(uint64_t) * ns, cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaMemcpyAsync(hc.data(), A.cell, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, ctx.stream));
    }
    CK(cudaMemcpyAsync(hv.data(), tmp, sizeof(double) * 6 * ns, cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    double* dst[6] = {x, y, u, v, w, m};
    int64_t o = 0;
    for (size_t i = 0; i < ns; ++i) {
        if (hc[i] < 0) continue;
        if (o >= n) return fail(ctx, UGKWP_ECUDA, "more live particle slots than the particle count");
        pid[o] = hp[i];
        cell[o] = hc[i];
        for (int k = 0; k < 6; ++k) dst[k][o] = hv[(size_t)k * ns + i];
        ++o;
    }
    if (o != n) return fail(ctx, UGKWP_ECUDA, "fewer live particle slots than the particle count");
    return UGKWP_OK;
}

ugkwp_status ugkwp_set_state(ugkwp_ctx* h, int64_t step, const double* W, const int64_t* wret, int64_t np,
                             const uint64_t* pid, const int32_t* cell, const double* x, const double* y, const double* u,
                             const double* v, const double* w, const double* m)
{
    if (!h || !W || !wret || np < 0) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    const int C = ctx.k.C;
    if (np > ctx.capacity || (ctx.k.wave_only && np > 0)) return fail(ctx, UGKWP_ELIMIT, "particle capacity exceeded");
    for (int64_t i = 0; i < np; ++i)
        if (cell[i] < 0 || cell[i] >= C) return fail(ctx, UGKWP_EINVAL, "particle cell index out of range");
    CK(cudaMemcpyAsync(ctx.d.W, W, sizeof(double) * 4 * C, cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaMemcpyAsync(ctx.d.wrt, wret, sizeof(int64_t) * 5 * C, cudaMemcpyHostToDevice, ctx.stream));
    long long st = step;
    CK(cudaMemcpyAsync(ctx.d.dstep, &st, sizeof st, cudaMemcpyHostToDevice, ctx.stream));
    int n32 = (int)np, zero = 0;
    const unsigned long long alive = (unsigned long long)np;
    CK(cudaMemcpyAsync(ctx.d.counts, &n32, sizeof(int), cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaMemcpyAsync(ctx.d.stats + 1, &alive, sizeof alive, cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaMemcpyAsync(ctx.d.bufsel, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx.stream));
    if (np > 0) {
        double* tmp = nullptr;
        int* tc = nullptr;
        unsigned long long* tp = nullptr;
        Tmp t1(ctx), t2(ctx), t3(ctx);
        CK(t1.get(&tmp, 6 * (size_t)np));
        CK(t2.get(&tc, (size_t)np));
        CK(t3.get(&tp, (size_t)np));
        const double* src[6] = {x, y, u, v, w, m};
        for (int k = 0; k < 6; ++k)
            CK(cudaMemcpyAsync(tmp + (size_t)k * np, src[k], sizeof(double) * np, cudaMemcpyHostToDevice, ctx.stream));
        CK(cudaMemcpyAsync(tc, cell, sizeof(int) * np, cudaMemcpyHostToDevice, ctx.stream));
        CK(cudaMemcpyAsync(tp, pid, sizeof(unsigned long long) * np, cudaMemcpyHostToDevice, ctx.stream));
        const int n = (int)np;
        if (ctx.k.prec == 0)
            k_put_particles<float><<<nblk(n, 256), 256, 0, ctx.stream>>>(ctx.d.pa32, n, tmp, tmp + np, tmp + 2 * np,
                                                                       tmp + 3 * np, tmp + 4 * np, tmp + 5 * np, tc, tp);
        else
            k_put_particles<double><<<nblk(n, 256), 256, 0, ctx.stream>>>(ctx.d.pa64, n, tmp, tmp + np, tmp + 2 * np,
                                                                        tmp + 3 * np, tmp + 4 * np, tmp + 5 * np, tc, tp);
        CK(cudaStreamSynchronize(ctx.stream));
    }
    CK(cudaStreamSynchronize(ctx.stream));
    ctx.step = step;
    return UGKWP_OK;
}

ugkwp_status ugkwp_get_tallies(ugkwp_ctx* h, int64_t* wm, int64_t* wpl, int64_t* wret, int64_t* cross, int64_t* wall,
                               int64_t* frec)
{
    if (!h) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    const size_t C = ctx.k.C, F = ctx.k.F;
    if (wm) CK(cudaMemcpyAsync(wm, ctx.d.wm, 8 * 5 * C, cudaMemcpyDeviceToHost, ctx.stream));
    if (wpl) CK(cudaMemcpyAsync(wpl, ctx.d.wpl, 8 * 5 * C, cudaMemcpyDeviceToHost, ctx.stream));
    if (wret) CK(cudaMemcpyAsync(wret, ctx.d.wrt, 8 * 5 * C, cudaMemcpyDeviceToHost, ctx.stream));
    if (wall && ctx.k.nwall) CK(cudaMemcpyAsync(wall, ctx.d.wallt, 8 * 3 * (size_t)ctx.k.nwall, cudaMemcpyDeviceToHost, ctx.stream));
    if (cross) {
        std::vector<unsigned int> cr(2 * F);
        CK(cudaMemcpyAsync(cr.data(), ctx.d.cross, 4 * 2 * F, cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaStreamSynchronize(ctx.stream));
        for (size_t i = 0; i < 2 * F; ++i) cross[i] = cr[i];
    }
    if (frec) {
        if (ctx.d.frec) CK(cudaMemcpyAsync(frec, ctx.d.frec, 8 * 4 * F, cudaMemcpyDeviceToHost, ctx.stream));
        else memset(frec, 0, 8 * 4 * F);
    }
    return check_device_error(ctx);
}

ugkwp_status ugkwp_get_cell_data(ugkwp_ctx* h, double* out)
{
    if (!h || !out) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    const int C = ctx.k.C;
    double* tmp = nullptr;
    Tmp t(ctx);
    CK(t.get(&tmp, 8 * (size_t)C));
    k_cell_data<<<nblk(C, 128), 128, 0, ctx.stream>>>(ctx.k, ctx.d, C, tmp);
    CK(cudaMemcpyAsync(out, tmp, sizeof(double) * 8 * C, cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    return UGKWP_OK;
}

ugkwp_status ugkwp_get_flux(ugkwp_ctx* h, double* flux)
{
    if (!h || !flux) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    CK(cudaMemcpyAsync(flux, ctx.d.flux, sizeof(double) * 4 * ctx.k.F, cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    return UGKWP_OK;
}

ugkwp_status ugkwp_get_geometry(ugkwp_ctx* h, double* dt, double* vol, int32_t* nfaces, int32_t* nwall)
{
    if (!h) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    if (dt) CK(cudaMemcpyAsync(dt, ctx.d.dt, sizeof(double) * ctx.k.C, cudaMemcpyDeviceToHost, ctx.stream));
    if (vol) CK(cudaMemcpyAsync(vol, ctx.d.vol, sizeof(double) * ctx.k.C, cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    if (nfaces) *nfaces = ctx.k.F;
    if (nwall) *nwall = ctx.k.nwall;
    return UGKWP_OK;
}

ugkwp_status ugkwp_fixed_exponents(ugkwp_ctx* h, int32_t* out)
{
    if (!h || !out) return UGKWP_EINVAL;
    out[0] = h->c.k.fx0; out[1] = h->c.k.fx1; out[2] = h->c.k.fx4;
    return UGKWP_OK;
}

ugkwp_status ugkwp_set_profiling(ugkwp_ctx* h, int32_t enable)
{
    if (!h) return UGKWP_EINVAL;
    h->c.profiling = enable ? 1 : 0;
    return UGKWP_OK;
}

ugkwp_status ugkwp_profile(ugkwp_ctx* h, double* ms, int64_t* steps)
{
    if (!h || !ms || !steps) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    CK(cudaStreamSynchronize(ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream2));
    for (int k = 0; k < kStages; ++k) ms[k] = 0.0;
    const size_t per = 2 * kStages, n = ctx.prof_events.size() / per;
    // stages in event-pair order: decompose, sample, particles, wave flux, sort, update
    const int order[kStages] = {0, 1, 2, 3, 4, 5};
    const int pair[kStages] = {0, 2, 4, 6, 8, 10};
    for (size_t i = 0; i < n; ++i)
        for (int k = 0; k < kStages; ++k) {
            float t = 0.0f;
            const int q = pair[order[k]];
            CK(cudaEventElapsedTime(&t, ctx.prof_events[i * per + q], ctx.prof_events[i * per + q + 1]));
            ms[k] += t;
        }
    for (cudaEvent_t e : ctx.prof_events) cudaEventDestroy(e);
    ctx.prof_events.clear();
    *steps = (int64_t)n;
    return UGKWP_OK;
}

struct ugkwp_batch {
    std::vector<ugkwp_ctx*> cases;
    std::vector<cudaStream_t> streams;
    cudaStream_t root = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraphExec_t graph = nullptr;
    std::string msg;
    // the persistent kernel (ugkwp_batch_create_persistent): device plan and control words, allocated through
    // the first case's allocator
    bool persistent = false;
    MkCase* mk_cases = nullptr;
    int4* mk_items = nullptr;
    int2* mk_dep = nullptr;
    int* mk_done = nullptr;
    MkCtl* mk_ctl = nullptr;
    int n_items = 0, grid = 0, ctas_per_sm = 0;
};

ugkwp_status ugkwp_batch_create(ugkwp_ctx* const* ctxs, int32_t n, void* stream, ugkwp_batch** out)
{
    if (!ctxs || n <= 0 || !out) return UGKWP_EINVAL;
    *out = nullptr;
    ugkwp_batch* b = new (std::nothrow) ugkwp_batch;
    if (!b) return UGKWP_ENOMEM;
    b->root = static_cast<cudaStream_t>(stream);
    auto bail = [&](ugkwp_status st) { ugkwp_batch_destroy(b); return st; };
    for (int32_t i = 0; i < n; ++i) {
        if (!ctxs[i]) return bail(UGKWP_EINVAL);
        for (int32_t j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return bail(UGKWP_EINVAL);
        b->cases.push_back(ctxs[i]);
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return bail(UGKWP_ECUDA);
        b->streams.push_back(s);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bail(UGKWP_ECUDA);
        b->joins.push_back(e);
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return bail(UGKWP_ECUDA);
    // one graph: fork every case from a capture stream, each case's step on its own streams, join all
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return bail(UGKWP_ECUDA);
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        cudaEventRecord(b->fork, cap);
        for (int32_t i = 0; i < n; ++i) {
            cudaStreamWaitEvent(b->streams[i], b->fork, 0);
            enqueue_step(b->cases[i]->c, b->streams[i], b->cases[i]->c.stream2, false);
            cudaEventRecord(b->joins[i], b->streams[i]);
            cudaStreamWaitEvent(cap, b->joins[i], 0);
        }
        ok = cudaStreamEndCapture(cap, &g) == cudaSuccess;
    }
    if (ok) ok = cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (!ok) return bail(UGKWP_ECUDA);
    *out = b;
    return UGKWP_OK;
}

ugkwp_status ugkwp_batch_step(ugkwp_batch* b, int32_t n_steps)
{
    if (!b || n_steps < 0) return UGKWP_EINVAL;
    // every case's previous work on its own stream completes first
    for (ugkwp_ctx* c : b->cases) {
        cudaEventRecord(b->fork, c->c.stream);
        cudaStreamWaitEvent(b->root, b->fork, 0);
    }
    for (int32_t k = 0; k < n_steps; ++k)
        if (cudaGraphLaunch(b->graph, b->root) != cudaSuccess) return UGKWP_ECUDA;
    cudaEventRecord(b->fork, b->root);
    for (ugkwp_ctx* c : b->cases) {
        cudaStreamWaitEvent(c->c.stream, b->fork, 0);
        c->c.step += n_steps;
    }
    return cudaGetLastError() == cudaSuccess ? UGKWP_OK : UGKWP_ECUDA;
}

void ugkwp_batch_destroy(ugkwp_batch* b)
{
    if (!b) return;
    if (b->root) cudaStreamSynchronize(b->root);
    else cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (!b->cases.empty()) {
        Ctx& c0 = b->cases[0]->c;
        raw_free(c0, b->mk_cases);
        raw_free(c0, b->mk_items);
        raw_free(c0, b->mk_dep);
        raw_free(c0, b->mk_done);
        raw_free(c0, b->mk_ctl);
    }
    delete b;
}

ugkwp_status ugkwp_batch_create_persistent(ugkwp_ctx* const* ctxs, int32_t n, void* stream, int32_t ctas_per_sm,
                                           ugkwp_batch** out)
{
    if (!ctxs || n <= 0 || n > kMkMaxCases || !out || (ctas_per_sm != 0 && ctas_per_sm != 4 && ctas_per_sm != 6))
        return UGKWP_EINVAL;
    *out = nullptr;
    int dev = -1;
    for (int32_t i = 0; i < n; ++i) {
        if (!ctxs[i]) return UGKWP_EINVAL;
        for (int32_t j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return UGKWP_EINVAL;
        const Ctx& c = ctxs[i]->c;
        // the kernel's scope: production precision, first order, the warp-staged transport with 128-particle
        // tiles, no per-stage profiling
        if (c.k.prec != 0 || c.k.order != 1 || c.transport != kTransportStaged || c.k.chunk != 128 || c.profiling)
            return UGKWP_EINVAL;
        if (i == 0) dev = c.device;
        else if (c.device != dev) return UGKWP_EINVAL;
    }
    ugkwp_batch* b = new (std::nothrow) ugkwp_batch;
    if (!b) return UGKWP_ENOMEM;
    b->root = static_cast<cudaStream_t>(stream);
    b->persistent = true;
    for (int32_t i = 0; i < n; ++i) b->cases.push_back(ctxs[i]);
    auto bail = [&](ugkwp_status st) { ugkwp_batch_destroy(b); return st; };
    Ctx& c0 = ctxs[0]->c;
    const int mb = ctas_per_sm ? ctas_per_sm : 4;
    int occ = 0;
    if ((mb == 4 ? mk_occupancy<4>(&occ) : mk_occupancy<6>(&occ)) != cudaSuccess || occ < 1) return bail(UGKWP_ECUDA);
    b->ctas_per_sm = std::min(occ, mb);
    b->grid = b->ctas_per_sm * c0.sms;
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return bail(UGKWP_ECUDA);
    // per case: its descriptor and stage sizes (particle count from the device)
    std::vector<MkCase> mc(n);
    for (int32_t i = 0; i < n; ++i) {
        Ctx& c = ctxs[i]->c;
        unsigned long long alive = 0;
        if (cudaMemcpyAsync(&alive, c.d.stats + 1, sizeof alive, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
            cudaStreamSynchronize(c.stream) != cudaSuccess)
            return bail(UGKWP_ECUDA);
        const long long np = std::max<long long>((long long)alive, (long long)c.k.n_ref * c.k.C);
        mc[i].K = c.k;
        mc[i].d = c.d;
        mk_plan_case(c, b->grid, np, mc[i]);
    }
    // the items in stage-major order, and each (case, stage)'s wait: the case's previous stage that runs
    std::vector<int4> items;
    std::vector<int2> dep((size_t)n * MS_COUNT, make_int2(-1, 0));
    std::vector<int> nitems((size_t)n * MS_COUNT, 0);
    for (int st = 0; st < MS_COUNT; ++st)
        for (int32_t i = 0; i < n; ++i) {
            const int nv = mc[i].nv[st];
            for (int b0 = 0; b0 < nv; b0 += kMkPer[st]) {
                items.push_back(make_int4(i, st, b0, std::min(nv, b0 + kMkPer[st])));
                nitems[(size_t)i * MS_COUNT + st]++;
            }
        }
    for (int32_t i = 0; i < n; ++i) {
        int prev = -1;
        for (int st = 0; st < MS_COUNT; ++st) {
            if (!mc[i].nv[st]) continue;
            if (prev >= 0) dep[(size_t)i * MS_COUNT + st] = make_int2(prev, nitems[(size_t)i * MS_COUNT + prev]);
            prev = st;
        }
    }
    b->n_items = (int)items.size();
    const MkCtl ctl0{0, 0, 0, -1, 2000000000ull, 0, 0};
    if (raw_alloc(c0, (void**)&b->mk_cases, sizeof(MkCase) * n) != cudaSuccess ||
        raw_alloc(c0, (void**)&b->mk_items, sizeof(int4) * items.size()) != cudaSuccess ||
        raw_alloc(c0, (void**)&b->mk_dep, sizeof(int2) * dep.size()) != cudaSuccess ||
        raw_alloc(c0, (void**)&b->mk_done, sizeof(int) * dep.size()) != cudaSuccess ||
        raw_alloc(c0, (void**)&b->mk_ctl, sizeof(MkCtl)) != cudaSuccess)
        return bail(UGKWP_ENOMEM);
    if (cudaMemcpyAsync(b->mk_cases, mc.data(), sizeof(MkCase) * n, cudaMemcpyHostToDevice, c0.stream) != cudaSuccess ||
        cudaMemcpyAsync(b->mk_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, c0.stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->mk_dep, dep.data(), sizeof(int2) * dep.size(), cudaMemcpyHostToDevice, c0.stream) !=
            cudaSuccess ||
        cudaMemsetAsync(b->mk_done, 0, sizeof(int) * dep.size(), c0.stream) != cudaSuccess ||
        cudaMemcpyAsync(b->mk_ctl, &ctl0, sizeof ctl0, cudaMemcpyHostToDevice, c0.stream) != cudaSuccess ||
        cudaStreamSynchronize(c0.stream) != cudaSuccess)
        return bail(UGKWP_ECUDA);
    // the launch, captured once
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return bail(UGKWP_ECUDA);
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        if (mb == 4)
            mk_launch<4>(b->grid, cap, b->mk_cases, b->mk_items, b->n_items, b->mk_dep, b->mk_done, (int)dep.size(),
                         b->mk_ctl, n);
        else
            mk_launch<6>(b->grid, cap, b->mk_cases, b->mk_items, b->n_items, b->mk_dep, b->mk_done, (int)dep.size(),
                         b->mk_ctl, n);
        ok = cudaStreamEndCapture(cap, &g) == cudaSuccess;
    }
    if (ok) ok = cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (!ok) return bail(UGKWP_ECUDA);
    *out = b;
    return UGKWP_OK;
}

ugkwp_status ugkwp_batch_set_wait_limit(ugkwp_batch* b, int64_t limit_ns, int32_t stall)
{
    if (!b || !b->persistent || limit_ns <= 0) return UGKWP_EINVAL;
    const unsigned long long lim = (unsigned long long)limit_ns;
    const int st = stall ? 1 : 0;
    cudaStream_t s = b->root;
    if (cudaMemcpyAsync(&b->mk_ctl->limit_ns, &lim, sizeof lim, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(&b->mk_ctl->stall, &st, sizeof st, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return UGKWP_ECUDA;
    return UGKWP_OK;
}

ugkwp_status ugkwp_batch_status(ugkwp_batch* b, int32_t* where)
{
    if (!b) return UGKWP_EINVAL;
    if (where) *where = -1;
    if (cudaStreamSynchronize(b->root) != cudaSuccess) return UGKWP_ECUDA;
    if (!b->persistent) return UGKWP_OK;
    MkCtl h;
    if (cudaMemcpy(&h, b->mk_ctl, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return UGKWP_ECUDA;
    if (!h.abort) return UGKWP_OK;
    if (where) *where = h.where;
    return UGKWP_ELIMIT;
}

ugkwp_status ugkwp_batch_plan(const ugkwp_batch* b, int32_t* out)
{
    if (!b || !out) return UGKWP_EINVAL;
    out[0] = b->persistent ? 1 : 0;
    out[1] = b->n_items;
    out[2] = b->grid;
    out[3] = b->ctas_per_sm;
    return UGKWP_OK;
}

namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, C, F, nwall, prec, wave_only;
    int64_t step, np;
    int32_t fx[3], pad;
};
}  // namespace

ugkwp_status ugkwp_save(ugkwp_ctx* h, const char* path)
{
    if (!h || !path) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    const int C = ctx.k.C, nw = ctx.k.nwall;
    const int64_t np = ugkwp_num_particles(h);
    if (np < 0) return fail(ctx, UGKWP_ECUDA, "reading the particle count");
    CkptHeader hd{};
    memcpy(hd.magic, "UGKWPCK1", 8);
    hd.version = 2; hd.C = C; hd.F = ctx.k.F; hd.nwall = nw; hd.prec = ctx.k.prec; hd.wave_only = ctx.k.wave_only;
    long long step = 0;
    CK(cudaMemcpyAsync(&step, ctx.d.dstep, sizeof step, cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    hd.step = step; hd.np = np; hd.fx[0] = ctx.k.fx0; hd.fx[1] = ctx.k.fx1; hd.fx[2] = ctx.k.fx4;
    std::vector<double> W(4 * (size_t)C), res(8), chi(C), ss(3 * (size_t)std::max(nw, 1));
    std::vector<long long> wr(5 * (size_t)C);
    unsigned long long st[16];
    CK(cudaMemcpyAsync(W.data(), ctx.d.W, 8 * W.size(), cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaMemcpyAsync(wr.data(), ctx.d.wrt, 8 * wr.size(), cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaMemcpyAsync(res.data(), ctx.d.res, 8 * 8, cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaMemcpyAsync(chi.data(), ctx.d.chi_ema, 8 * (size_t)C, cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaMemcpyAsync(ss.data(), ctx.d.surf_sum, 8 * ss.size(), cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaMemcpyAsync(st, ctx.d.stats, sizeof st, cudaMemcpyDeviceToHost, ctx.stream));
    double mon[8];
    CK(cudaMemcpyAsync(mon, ctx.d.mon, sizeof mon, cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    std::vector<uint64_t> pid(np > 0 ? np : 1);
    std::vector<int32_t> cell(np > 0 ? np : 1);
    std::vector<double> pv(6 * (size_t)(np > 0 ? np : 1));
    if (np > 0) {
        ugkwp_status e = ugkwp_get_particles(h, np, pid.data(), cell.data(), pv.data(), pv.data() + np,
                                             pv.data() + 2 * np, pv.data() + 3 * np, pv.data() + 4 * np, pv.data() + 5 * np);
        if (e) return e;
    }
    FILE* f = fopen(path, "wb");
    if (!f) return fail(ctx, UGKWP_EINVAL, "cannot open the checkpoint file for writing");
    bool ok = fwrite(&hd, sizeof hd, 1, f) == 1 && fwrite(W.data(), 8, W.size(), f) == W.size() &&
              fwrite(wr.data(), 8, wr.size(), f) == wr.size() && fwrite(res.data(), 8, 8, f) == 8 &&
              fwrite(chi.data(), 8, chi.size(), f) == chi.size() && fwrite(ss.data(), 8, ss.size(), f) == ss.size() &&
              fwrite(st, sizeof st, 1, f) == 1 && fwrite(mon, sizeof mon, 1, f) == 1;
    if (ok && np > 0)
        ok = fwrite(pid.data(), 8, np, f) == (size_t)np && fwrite(cell.data(), 4, np, f) == (size_t)np &&
             fwrite(pv.data(), 8, 6 * np, f) == (size_t)(6 * np);
    ok = (fclose(f) == 0) && ok;
    return ok ? UGKWP_OK : fail(ctx, UGKWP_EINVAL, "writing the checkpoint file failed");
}

ugkwp_status ugkwp_load(ugkwp_ctx* h, const char* path)
{
    if (!h || !path) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    const int C = ctx.k.C, nw = ctx.k.nwall;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(ctx, UGKWP_EINVAL, "cannot open the checkpoint file");
    CkptHeader hd{};
    bool ok = fread(&hd, sizeof hd, 1, f) == 1 && memcmp(hd.magic, "UGKWPCK1", 8) == 0 && hd.version == 2 &&
              hd.C == C && hd.F == ctx.k.F && hd.nwall == nw && hd.prec == ctx.k.prec &&
              hd.fx[0] == ctx.k.fx0 && hd.fx[1] == ctx.k.fx1 && hd.fx[2] == ctx.k.fx4 && hd.np >= 0 &&
              hd.np <= ctx.capacity;
    if (!ok) { fclose(f); return fail(ctx, UGKWP_EINVAL, "checkpoint does not match this context"); }
    const int64_t np = hd.np;
    std::vector<double> W(4 * (size_t)C), res(8), chi(C), ss(3 * (size_t)std::max(nw, 1));
    std::vector<long long> wr(5 * (size_t)C);
    unsigned long long st[16];
    double mon[8];
    std::vector<uint64_t> pid(np > 0 ? np : 1);
    std::vector<int32_t> cell(np > 0 ? np : 1);
    std::vector<double> pv(6 * (size_t)(np > 0 ? np : 1));
    ok = fread(W.data(), 8, W.size(), f) == W.size() && fread(wr.data(), 8, wr.size(), f) == wr.size() &&
         fread(res.data(), 8, 8, f) == 8 && fread(chi.data(), 8, chi.size(), f) == chi.size() &&
         fread(ss.data(), 8, ss.size(), f) == ss.size() && fread(st, sizeof st, 1, f) == 1 &&
         fread(mon, sizeof mon, 1, f) == 1;
    if (ok && np > 0)
        ok = fread(pid.data(), 8, np, f) == (size_t)np && fread(cell.data(), 4, np, f) == (size_t)np &&
             fread(pv.data(), 8, 6 * np, f) == (size_t)(6 * np);
    fclose(f);
    if (!ok) return fail(ctx, UGKWP_EINVAL, "truncated checkpoint file");
    ugkwp_status e = ugkwp_set_state(h, hd.step, W.data(), reinterpret_cast<const int64_t*>(wr.data()), np,
                                     pid.data(), cell.data(), pv.data(), pv.data() + np, pv.data() + 2 * np,
                                     pv.data() + 3 * np, pv.data() + 4 * np, pv.data() + 5 * np);
    if (e) return e;
    CK(cudaMemcpyAsync(ctx.d.res, res.data(), 8 * 8, cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaMemcpyAsync(ctx.d.chi_ema, chi.data(), 8 * (size_t)C, cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaMemcpyAsync(ctx.d.surf_sum, ss.data(), 8 * ss.size(), cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaMemcpyAsync(ctx.d.stats, st, sizeof st, cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaMemcpyAsync(ctx.d.mon, mon, sizeof mon, cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    return UGKWP_OK;
}

const char* ugkwp_last_error(const ugkwp_ctx* h)
{
    return h ? h->c.msg.c_str() : "null context";
}

}  // extern "C"

// ---- ugkwp_get_field_noalloc: ugkwp_get_field without any allocation ------------------------------------
// For callers that must not allocate device memory: cudaMalloc and cudaFree synchronise the whole device,
// so a monitor thread that samples a running case while other cases run on other streams (the batched
// launch) would stall all of them, and a run whose particle buffers were sized to fill device memory has
// no room left for a temporary. The W^p conversion goes through a fixed scratch array in device memory
// instead of a per-call temporary; nothing else differs from ugkwp_get_field (same kernel, same values).
//
// Scratch: 4 doubles per cell for at most kNoAllocMaxCells cells (3 MiB per device). Nothing in it needs to
// start at zero: every element read is first written by the same call. All calls on one device share it, so
// calls that overlap in time (from several host threads, or for several contexts on one device) race on it:
// callers serialise them. The scratch address is looked up once per device (cudaGetSymbolAddress) on the
// first call with a non-NULL Wp on that device; make that first call before any stream capture begins. The
// context's device must be the current one (the scratch is the current device's).
#include <mutex>

namespace {
constexpr int kNoAllocMaxCells = 98304;
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[4 * kNoAllocMaxCells];

extern "C" ugkwp_status ugkwp_get_field_noalloc(ugkwp_ctx* h, double* W, double* Wp)
{
    if (!h || !W) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    const int C = ctx.k.C;
    // every check comes before the first copy is queued, so an error return leaves nothing in flight
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != ctx.device)
        return fail(ctx, UGKWP_EINVAL, "ugkwp_get_field_noalloc: the context's device is not the current device");
    double* scratch = nullptr;
    if (Wp) {
        if (C > kNoAllocMaxCells)
            return fail(ctx, UGKWP_EINVAL, "ugkwp_get_field_noalloc: the mesh has more than 98304 cells (its scratch limit)");
        if (dev < 0 || dev >= kNoAllocMaxDevices)
            return fail(ctx, UGKWP_EINVAL, "ugkwp_get_field_noalloc: device ordinal beyond its table of 64");
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fail(ctx, UGKWP_ECUDA, "ugkwp_get_field_noalloc: cudaGetSymbolAddress of the scratch failed");
            g_noalloc_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    // from here on a failure waits for the copies already queued before it returns, so that the caller may
    // reuse its host buffers at once
    const auto queued_fail = [&](cudaError_t e, const char* what) {
        cudaStreamSynchronize(ctx.stream);
        ctx.msg = std::string(what) + ": " + cudaGetErrorString(e);
        return UGKWP_ECUDA;
    };
    cudaError_t e = cudaMemcpyAsync(W, ctx.d.W, sizeof(double) * 4 * C, cudaMemcpyDeviceToHost, ctx.stream);
    if (e != cudaSuccess) return queued_fail(e, "ugkwp_get_field_noalloc: W copy");
    if (Wp) {
        k_wp_field<<<nblk(C, 128), 128, 0, ctx.stream>>>(ctx.d, C, ctx.k.fx0, ctx.k.fx1, ctx.k.fx4, scratch);
        e = cudaGetLastError();
        if (e != cudaSuccess) return queued_fail(e, "ugkwp_get_field_noalloc: W^p conversion launch");
        e = cudaMemcpyAsync(Wp, scratch, sizeof(double) * 4 * C, cudaMemcpyDeviceToHost, ctx.stream);
        if (e != cudaSuccess) return queued_fail(e, "ugkwp_get_field_noalloc: W^p copy");
    }
    return check_device_error(ctx);
}

// ---- launch parameters and their autotuner ----------------------------------------------------------------
// The particle kernels' launch shape (chunk of particles a warp claims, blocks per SM) and the counting-sort
// interval change only the speed of a step: chunks and the sort reorder particles, and every result is an
// integer sum or a per-particle / per-face quantity, so the state after a step is the same.
namespace {
ugkwp_status apply_launch(Ctx& ctx, int chunk, int bps, int sort_every, int transport)
{
    if (transport) {
        if (transport != kTransportWarp && transport != kTransportStaged)
            return fail(ctx, UGKWP_EINVAL, "transport kernel: 1 (warp-chunked) or 2 (warp-staged)");
        if (transport == kTransportStaged && ctx.k.prec != 0)
            return fail(ctx, UGKWP_EINVAL, "the warp-staged transport kernel serves the production precision only");
        ctx.transport = transport;
    }
    if (chunk) {
        if (chunk < 32 || chunk > 8192 || chunk % 32) return fail(ctx, UGKWP_EINVAL, "chunk: a multiple of 32 in [32, 8192]");
        ctx.k.chunk = chunk;
    }
    if (bps) {
        if (bps < 1 || bps > 16) return fail(ctx, UGKWP_EINVAL, "blocks per SM: 1 to 16");
        ctx.grid_particles = ctx.sms * bps;
    }
    if (sort_every) {
        if (sort_every < 1 || sort_every > 64) return fail(ctx, UGKWP_EINVAL, "sort interval: 1 to 64 steps");
        ctx.k.sort_every = sort_every;
    }
    if (ctx.graph) {   // the captured step holds the old constants
        cudaGraphExecDestroy(ctx.graph);
        ctx.graph = nullptr;
    }
    return UGKWP_OK;
}
}  // namespace

extern "C" ugkwp_status ugkwp_set_launch(ugkwp_ctx* h, int32_t chunk, int32_t blocks_per_sm, int32_t sort_every,
                                        int32_t transport)
{
    if (!h) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    CK(cudaStreamSynchronize(ctx.stream));
    return apply_launch(ctx, chunk, blocks_per_sm, sort_every, transport);
}

extern "C" ugkwp_status ugkwp_get_launch(ugkwp_ctx* h, int32_t* out)
{
    if (!h || !out) return UGKWP_EINVAL;
    const Ctx& ctx = h->c;
    out[0] = ctx.k.chunk;
    out[1] = ctx.grid_particles / ctx.sms;
    out[2] = ctx.k.sort_every;
    out[3] = ctx.transport;
    return UGKWP_OK;
}

extern "C" ugkwp_status ugkwp_autotune(ugkwp_ctx* h, int32_t steps, int32_t* best, double* best_ms)
{
    if (!h || steps < 1) return UGKWP_EINVAL;
    Ctx& ctx = h->c;
    if (ctx.k.wave_only) {   // no particle kernels to tune
        if (best) ugkwp_get_launch(h, best);
        if (best_ms) *best_ms = 0.0;
        return UGKWP_OK;
    }
    // candidates: the warp-staged kernel (production precision; 64-particle tiles at 6 or 8 CTAs per SM,
    // 128-particle tiles at 4, 6 or 8) and the warp-chunked kernel with chunk {128, 256} x blocks per SM {4, 6, 8}, each with sort interval {8, 16, 32}
    struct Cand { int chunk, bps, sort, transport; };
    std::vector<Cand> cands;
    for (int so : {8, 16, 32}) {
        if (ctx.k.prec == 0) {
            cands.push_back({64, 6, so, kTransportStaged});
            cands.push_back({64, 8, so, kTransportStaged});
            cands.push_back({128, 4, so, kTransportStaged});
            cands.push_back({128, 6, so, kTransportStaged});
            cands.push_back({128, 8, so, kTransportStaged});
        }
        for (int ch : {128, 256})
            for (int bp : {4, 6, 8}) cands.push_back({ch, bp, so, kTransportWarp});
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double bms = 1e300;
    int b[4] = {ctx.k.chunk, ctx.grid_particles / ctx.sms, ctx.k.sort_every, ctx.transport};
    ugkwp_status st = UGKWP_OK;
    for (const Cand& cd : cands) {
        if (st != UGKWP_OK) break;
        CK(cudaStreamSynchronize(ctx.stream));
        if ((st = apply_launch(ctx, cd.chunk, cd.bps, cd.sort, cd.transport)) != UGKWP_OK) break;
        const int so = cd.sort;
        // untimed steps (graph capture, then up to the next sort step), then whole sort periods
        const int lead = (int)((so - 1 - ctx.step % so + so) % so) + 1;
        if ((st = ugkwp_step(h, lead)) != UGKWP_OK) break;
        const int n = ((steps + so - 1) / so) * so;
        CK(cudaEventRecord(e0, ctx.stream));
        if ((st = ugkwp_step(h, n)) != UGKWP_OK) break;
        CK(cudaEventRecord(e1, ctx.stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms / n < bms) {
            bms = ms / n;
            b[0] = ctx.k.chunk; b[1] = ctx.grid_particles / ctx.sms; b[2] = so; b[3] = cd.transport;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != UGKWP_OK) return st;
    if ((st = check_device_error(ctx)) != UGKWP_OK) return st;
    if ((st = apply_launch(ctx, b[0], b[1], b[2], b[3])) != UGKWP_OK) return st;
    if (best) { best[0] = b[0]; best[1] = b[1]; best[2] = b[2]; best[3] = b[3]; }
    if (best_ms) *best_ms = bms;
    return UGKWP_OK;
}
