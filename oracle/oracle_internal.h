/* ORACLE (test infrastructure only): internal declarations shared by the oracle's own translation units. */
#ifndef ORACLE_INTERNAL_H
#define ORACLE_INTERNAL_H
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ELIMIT = 4, OR_ENONPHYS = 5, OR_EOVERFLOW = 6 };
enum { OR_BC_WALL = 1, OR_BC_FARFIELD = 2, OR_BC_FIXED = 3, OR_BC_SYMMETRY = 4, OR_BC_PERIODIC = 5 };

#define OR_R 0.5                 /* gas constant in the reference units (2 R T_inf = 1) */
#define OR_MAX_ITERS 256         /* face crossings + wall hits per particle per step */
#define OR_MAX_NEW 2047          /* new particles per cell per step (11-bit index in the id) */
#define OR_RHO_FLOOR 1e-12       /* vacuum floor of the cell density (units of rho_inf) */


typedef struct {
    double x, y, u, v, w, m;     /* FP32-representable values in production emulation */
    int32_t cell;
    uint64_t pid;
    /* per-step scratch */
    double tf;                   /* free-flight time; for a particle entering from a ghost, its time left */
    int32_t is_new, collide, alive, iters, entry0;   /* entry0: local face it entered through, or -1 */
} or_particle;

struct oracle_ctx {
    /* configuration */
    int dim, ni, nj, periodic_j, C, F;
    int prec, wave_only, record_faces, gts, n_ref, order;
    double emx_cutoff;                           /* cells with e^{-x} below it sample no new particles */
    uint64_t seed;
    uint32_t case_id;
    int64_t step;
    double Kn, Ma, Tw, cfl, omega, Pr, mu_inf, U_inf;
    double ws;                                   /* Maxwell wall: specular fraction 1 - alpha */
    double W_inf[4], W_fix[4];
    int fx[5];                                   /* fixed-point exponents: mass, momentum, energy; second and
                                                  * third velocity moments (Shakhov heat flux, Pr != 1) */
    double T_cap, U_cap, T_min;                  /* realizability bounds of a cell state */
    /* cells */
    double *vol, *inv_vol, *xc, *yc;
    int *nfc;
    int *cface, *csgn, *cnbr, *cnk, *cbc;        /* [4C] */
    double *cnx, *cny, *cd, *cshift;             /* [4C] outward normal, plane offset, periodic shift */
    double *cvx, *cvy;                           /* [4C] vertices, counter-clockwise */
    double *xl, *xr;                             /* 1-D cell ends */
    /* faces */
    int *fL, *fR, *fbc, *fwall;
    double *fnx, *fny, *fs, *fdL, *fdR, *finv_s;
    double *fax, *fay, *fex, *fey;               /* face start vertex a and edge b - a (1-D: the face point) */
    int n_inj;                                   /* far-field and fixed faces, in face order: ghost particle sources */
    int *inj_face, *inj_k;                       /* their face ids and local index in the fluid cell */
    int* inj_n;                                  /* per source: particles sampled this step */
    double *inj_m, *inj_u, *inj_v, *inj_sig, *inj_D;   /* per source: mass, ghost U, V, sqrt(RT), slab depth */
    int nwall;
    int *wall_face;
    /* time steps */
    double *dt, *ratio;                          /* dt[C]; ratio[4C] = dt[nbr] / dt[c] */
    double dtG;
    /* state */
    double *W;                                   /* [4C] */
    int64_t *wret_prev;                          /* [5C] retained tally of the previous step */
    /* per-step cell data */
    double *tau, *xr_t, *emx, *Wp, *Wh, *mnew, *co;   /* co: [7C] normalised coefficients */
    double* samp;                                /* [3C] U_i, V_i, R T_i of the sampling (cell state) */
    double* grad;                                /* [16C] order 2: limited gradients (d/dx, d/dy) of the 4
                                                  * components of W, then of W^h (S6) */
    int64_t* whq;                                /* [9C] retained particles: m (1, u, v, uu, uv, vv, q, uq, vq),
                                                  * q = |u|^2, fixed point (Pr != 1) */
    double* hq;                                  /* [3C] A-R weights a_x, a_y and bound M (Pr != 1) */
    double m2RTw, sig_w;                         /* -2 R T_w and sqrt(R T_w) */
    int *nhp;
    int64_t *nhp_off;
    /* tallies */
    int64_t *wm, *wpl, *wrt, *cross, *wallt;
    int64_t* frec;                               /* [4F] side-recorded crossing masses of this step (S33) */
    double *flux;                                /* [4F] */
    /* particles */
    int64_t np, cap;
    or_particle* p;
    /* diagnostics */
    double res[4];
    double* chi_ema;
    double *surf_sum, *surf_last;
    int64_t nsurf;
    double mon[8];                               /* C_d, C_H, stagnation C_p and C_Q, then their EMAs */
    int stag[2];                                 /* wall faces of the stagnation point (-1: none) */
    int64_t stats[11];                           /* [8]: cells set to the vacuum floor in the last step,
                                                  * [9]: A-R samplings that fell back to the Maxwellian,
                                                  * [10]: particles entering from far-field / fixed ghosts */
    int err;
    char msg[256];
};
typedef struct oracle_ctx or_ctx;

/* rng */
void   or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void   or_draw(const or_ctx* cx, uint64_t pid, uint32_t draw, uint32_t out[4]);
float  or_u01f(uint32_t w);
double or_u01d(uint32_t lo, uint32_t hi);
void   or_uniforms_f(const or_ctx* cx, uint64_t pid, uint32_t base, int n, float* u);
void   or_uniforms_d(const or_ctx* cx, uint64_t pid, uint32_t base, int n, double* u);
/* deterministic math */
float  or_logf(float x);
double or_logd(double x);
double or_expd(double x);
double or_erfcd(double x);
float  or_expf(float x);
double or_powd(double x, double y);
void   or_sincos2pif(float u, float* s, float* c);
void   or_sincos2pid(double u, double* s, double* c);
/* particles (float and double instantiations) */
void or_particles_step_f32(or_ctx* cx);
void or_particles_step_f64(or_ctx* cx);
void or_heat_tally_f32(or_ctx* cx);
void or_heat_tally_f64(or_ctx* cx);
int or_new_velocity_f32(const or_ctx* cx, uint64_t pid, int shakhov, float ax, float ay, float M, float z[3]);
int or_new_velocity_f64(const or_ctx* cx, uint64_t pid, int shakhov, double ax, double ay, double M, double z[3]);
void or_set_error(or_ctx* cx, int code, const char* msg);

/* Philox draw layout: the first counter word of each draw group */
#define OR_DRAW_POS 0u
#define OR_DRAW_VEL 2u
#define OR_DRAW_TF 5u
#define OR_DRAW_WALL(h) (8u + 2u * (uint32_t)(h))
#define OR_DRAW_AR(a) (1024u + 4u * (uint32_t)(a))   /* Shakhov A-R attempt a: proposal +0, +1; acceptance +2 */
#define OR_AR_ATTEMPTS 64

#endif
