/* ORACLE (test infrastructure only). Plain, slow CPU restatement of one UGKWP-LTS steady-iteration step,
 * used by the tests, the smoke check and the CPU-baseline leg of the benchmark to check the CUDA library.
 * Nothing in the product path may include, link or call it.
 *
 * The API mirrors the library's C ABI with an `oracle_` prefix; the structs are declared here separately
 * (same field order) so that the two implementations share no header.
 *
 * Status codes: 0 ok, 1 invalid argument, 2 out of memory, 4 limit hit (crossing cap, particle capacity,
 * more than 2047 new particles in a cell), 5 non-physical state, 6 fixed-point tally overflow.
 */
#ifndef ORACLE_UGKWP_H
#define ORACLE_UGKWP_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_ctx oracle_ctx;

typedef struct {
    int32_t ni, nj;          /* cells, i fastest */
    int32_t dim;             /* 1: line (nj = 1, only i-faces); 2: quadrilaterals */
    int32_t periodic_j;      /* 2-D: row j = nj wraps onto row 0 */
    const double* xv;        /* (ni+1)*(nj+1) vertex coordinates, index i + (ni+1) j */
    const double* yv;
    const int32_t* bc_imin;  /* nj boundary tags of the i = 0 faces */
    const int32_t* bc_imax;  /* nj tags of the i = ni faces */
    const int32_t* bc_jmin;  /* ni tags of the j = 0 faces (2-D, not periodic) */
    const int32_t* bc_jmax;  /* ni tags of the j = nj faces */
} oracle_mesh;

/* Unstructured mesh of triangles and convex quadrilaterals. Local face k of a cell is its edge from vertex k
 * to vertex k + 1 (mod 3 or 4); faces are numbered in order of first appearance over the cells and their
 * edges, the first cell naming an edge is its L side and the edge keeps that cell's direction. */
typedef struct {
    int32_t n_vertices, n_cells;
    const double* xv;          /* n_vertices coordinates */
    const double* yv;
    const int32_t* cells;      /* 4 vertex indices per cell, counter-clockwise; -1 in the fourth: a triangle */
    int32_t n_boundary;        /* edges of one cell, each tagged exactly once */
    const int32_t* boundary;   /* 3 per boundary edge: vertex, vertex (either order), tag (wall, far field,
                                * fixed or symmetry) */
} oracle_umesh;

typedef struct {
    double omega, Pr;
    double wall_specular;    /* Maxwell wall: fraction 1 - alpha reflected specularly; 0 = fully diffuse */
} oracle_gas;

typedef struct {
    uint64_t seed;
    uint32_t case_id;
    int32_t n_ref;
    int32_t precision;       /* 0: production emulation (FP32 particles; FP32 tau, e^{-x} away from walls at
                              * first order); 1: all FP64 */
    int32_t wave_only;       /* 1: no particles (deterministic GKS limit) */
    int32_t record_faces;    /* 1: per-face side-recorded crossing masses of each step (S33): frec[4 f + 2 d]
                              * the masses before, frec[4 f + 2 d + 1] after the scaling, d = 0 for L -> R,
                              * 1 for R -> L, as fixed-point integers of the mass exponent */
    int32_t capacity;        /* particle capacity; 0 = 4 * n_ref * cells */
    double ghost_state[4];   /* (rho, U, V, T) of BC_FIXED ghosts */
    int32_t order;           /* 2: second-order reconstruction of W and W^h (S6); 0 or 1: first order */
    double emx_cutoff;       /* cells with e^{-dt_i/tau_i} below it sample no new particles (0: off) */
} oracle_opts;

int  oracle_create(const oracle_mesh* mesh, const oracle_gas* gas, double Kn, double Ma, double Tw,
                   double cfl, int32_t gts, const oracle_opts* opts, oracle_ctx** out);
int  oracle_create_unstructured(const oracle_umesh* mesh, const oracle_gas* gas, double Kn, double Ma, double Tw,
                                double cfl, int32_t gts, const oracle_opts* opts, oracle_ctx** out);
void oracle_destroy(oracle_ctx* cx);
int  oracle_step(oracle_ctx* cx, int32_t n_steps);
int  oracle_set_field(oracle_ctx* cx, const double* prim);          /* 4 per cell: rho, U, V, T */
int  oracle_get_field(oracle_ctx* cx, double* W, double* Wp);       /* 4 per cell each; Wp nullable */
int  oracle_residual(oracle_ctx* cx, double* out);                  /* [8]: freestream-normalised, raw */
int  oracle_surface(oracle_ctx* cx, double* p, double* tau, double* q, int32_t n_wall, int32_t averaged);
/* monitored wall loads of the last step: C_d, C_H, stagnation C_p, C_Q (NaN without a stagnation point), then
 * their EMAs (alpha = 2/1001) from the first step on */
int  oracle_monitors(oracle_ctx* cx, double* out);
int  oracle_reset_surface(oracle_ctx* cx);
/* building block: n new-particle normal triples z[3n] of particle ids pid0 + k drawn for a Shakhov cell with
 * acceptance-rejection weights (ax, ay, M) (see shakhov_weights); returns the fallback count */
int64_t oracle_ar_sample(int32_t precision, uint64_t seed, uint32_t case_id, int64_t step, uint64_t pid0, int32_t n,
                         double ax, double ay, double M, double* z);
int  oracle_stats(oracle_ctx* cx, int64_t* out);                    /* [11] */
int64_t oracle_num_particles(oracle_ctx* cx);
int  oracle_get_particles(oracle_ctx* cx, int64_t cap, uint64_t* pid, int32_t* cell, double* x, double* y,
                          double* u, double* v, double* w, double* m);
int  oracle_set_state(oracle_ctx* cx, int64_t step, const double* W, const int64_t* wret, int64_t np,
                      const uint64_t* pid, const int32_t* cell, const double* x, const double* y,
                      const double* u, const double* v, const double* w, const double* m);
/* geometry: per cell (x_c, y_c, area), per face (L, R, tag) and (n_x, n_y, length, d_L, d_R); each nullable */
int  oracle_get_mesh(oracle_ctx* cx, double* cells, int32_t* faces, double* fgeo);
int  oracle_set_time_steps(oracle_ctx* cx, const double* dt);       /* C local steps, each > 0 (Sec. IV A) */
int  oracle_get_tallies(oracle_ctx* cx, int64_t* wm, int64_t* wpl, int64_t* wret, int64_t* cross,
                        int64_t* wall, int64_t* frec);
int  oracle_get_cell_data(oracle_ctx* cx, double* out);            /* [8 per cell] see oracle_core.c */
int  oracle_get_gradients(oracle_ctx* cx, double* out);             /* [16 per cell], order 2, see oracle_core.c */
int  oracle_get_shakhov(oracle_ctx* cx, double* out);               /* [3 per cell]: a_x, a_y, M of the last step */
void oracle_wall_flux_test(double Tw, double ws, const double* WL, const double* WhL, const double* cL, double frL,
                           double* F);                               /* wall face flux, face frame (pins) */
int  oracle_get_flux(oracle_ctx* cx, double* flux);                 /* [4 per face], global frame */
int  oracle_get_geometry(oracle_ctx* cx, double* dt, double* vol, int32_t* nfaces, int32_t* nwall);
int  oracle_fixed_exponents(oracle_ctx* cx, int32_t* out);          /* [3] mass, momentum, energy */
const char* oracle_last_error(oracle_ctx* cx);

/* building blocks exported for the pins */
void   oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out);
float  oracle_logf(float x);
double oracle_logd(double x);
double oracle_expd(double x);
float  oracle_expf(float x);
void   oracle_sincos2pif(float u, float* s, float* c);
void   oracle_sincos2pid(double u, double* s, double* c);
void   oracle_coeffs(double dt, double tau, double* out);           /* [7] */
void   oracle_face_flux_test(const double* WL, const double* WR, const double* WhL, const double* WhR,
                             const double* cL, const double* cR, double dL, double dR, double Pr,
                             double* F, double* W0, double* aL, double* aR, double* A);
double oracle_mu_inf(double Kn, double omega);
void   oracle_balance_condition(int32_t M, const double* dtL, const double* dtR, double* out);

#ifdef __cplusplus
}
#endif
#endif
