// Learned warm start: a coordinate MLP that maps a cell centroid and the case conditions (x, y, Kn, Ma, T_w)
// to an initial macroscopic field (log rho, u / U_inf, v / U_inf, log T). It changes only the field the
// steady LTS iteration (Sec. III C, Sec. IV B) starts from; the local time steps, fixed at creation from the
// freestream, and the iteration itself are untouched, so the converged state is the method's own.
//
// Network: n_features inputs, `depth` hidden SiLU layers of `width` units, a linear output layer. Weights are
// kept in FP32 (master copy, Adam state) and used in every product as BF16 values (round to nearest even);
// activations and accumulation are FP32. Activations are point-major [n][width].
//
// Products run on the tensor cores (mma.sync, BF16 operands with FP32 operands split into two BF16 terms,
// FP32 accumulation; 64 x 64 output tiles). Weight gradients split the point range over blockIdx.z into partial sums that a second kernel adds
// in a fixed order, so gradients are deterministic run to run.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>
#include "ugkwp_internal.h"

namespace {

constexpr int kTile = 64;
constexpr int kMaxSplit = 32;          // partial sums of a weight gradient
constexpr int kPointsPerSplit = 512;
constexpr int kFeatUsed = 37;          // 32 Fourier features, x^, y^, Kn, Ma, T_w

// The three products run on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation). A block
// computes a 64 x 64 output tile with 4 warps (2 x 2, 32 x 32 each: 2 x 4 MMA tiles), stepping the contraction
// 16 at a time through shared memory. Weights are BF16 values already, so they enter exactly; an FP32 operand
// (activations, back-propagated gradients, inputs) is split as v = hi + lo with hi = bf16(v), lo =
// bf16(v - hi), which keeps about 16 bits of its significand (relative error below 2^-17). Products with a
// weight take hi*W + lo*W; the weight gradient, whose operands are both FP32, takes hi*hi + hi*lo + lo*hi
// (the dropped lo*lo is below 2^-16 of the product). Every product of two BF16 values is exact in FP32, so
// the results stay within a few FP32 roundings of the FP32 products with BF16 weights that the network
// defines.
constexpr int kMmaThreads = 128;
constexpr int kKs = 16;              // contraction step
constexpr int kSmStride = kKs + 8;   // shared row stride in BF16 elements (48 B: conflict-free fragment loads)

struct MmaTiles {
    __nv_bfloat16 a_hi[kTile][kSmStride], a_lo[kTile][kSmStride];
    __nv_bfloat16 b_hi[kTile][kSmStride], b_lo[kTile][kSmStride];
};

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Stage rows r0..r0+63, contraction k0..k0+15 of an operand: thread t loads row t / 2, 8 consecutive k
// (zero outside the bounds), splits them and stores 16 bytes into each of hi and lo (lo skipped when null).
template <class Get>
__device__ __forceinline__ void stage_tile(Get get, __nv_bfloat16 (*hi)[kSmStride], __nv_bfloat16 (*lo)[kSmStride])
{
    const int r = threadIdx.x >> 1, kk = (threadIdx.x & 1) * 8;
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) split_bf16(get(r, kk + q), h[q], l[q]);
    *reinterpret_cast<uint4*>(&hi[r][kk]) = *reinterpret_cast<const uint4*>(h);
    if (lo) *reinterpret_cast<uint4*>(&lo[r][kk]) = *reinterpret_cast<const uint4*>(l);
}

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// acc += A(64 x 16) B(64 x 16)^T from the staged tiles: 2 terms (B exact) or 3 (both split)
__device__ __forceinline__ void mma_step(const MmaTiles& S, bool b_split, float (&acc)[2][4][4])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = (warp >> 1) * 32, n0 = (warp & 1) * 32;
    uint32_t ah[2][4], al[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int r = m0 + mt * 16 + g;
        ah[mt][0] = lds32(&S.a_hi[r][2 * t]);     ah[mt][1] = lds32(&S.a_hi[r + 8][2 * t]);
        ah[mt][2] = lds32(&S.a_hi[r][2 * t + 8]); ah[mt][3] = lds32(&S.a_hi[r + 8][2 * t + 8]);
        al[mt][0] = lds32(&S.a_lo[r][2 * t]);     al[mt][1] = lds32(&S.a_lo[r + 8][2 * t]);
        al[mt][2] = lds32(&S.a_lo[r][2 * t + 8]); al[mt][3] = lds32(&S.a_lo[r + 8][2 * t + 8]);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int c = n0 + nt * 8 + g;
        const uint32_t bh0 = lds32(&S.b_hi[c][2 * t]), bh1 = lds32(&S.b_hi[c][2 * t + 8]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            mma_bf16(acc[mt][nt], al[mt], bh0, bh1);
            if (b_split) mma_bf16(acc[mt][nt], ah[mt], lds32(&S.b_lo[c][2 * t]), lds32(&S.b_lo[c][2 * t + 8]));
            mma_bf16(acc[mt][nt], ah[mt], bh0, bh1);
        }
    }
}

// the output element (row, col) of accumulator register q of MMA tile (mt, nt) of this thread
__device__ __forceinline__ void acc_coord(int mt, int nt, int q, int& row, int& col)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    row = (warp >> 1) * 32 + mt * 16 + (lane >> 2) + (q >> 1) * 8;
    col = (warp & 1) * 32 + nt * 8 + (lane & 3) * 2 + (q & 1);
}

// Y[n][N] = act(X[rows][K] W^T + b); pre-activations kept in Z for the backward pass. rows == nullptr: rows 0..n-1
__global__ void __launch_bounds__(kMmaThreads) k_linear_fwd(const float* __restrict__ X, const int* __restrict__ rows,
                                                            const __nv_bfloat16* __restrict__ W,
                                                            const float* __restrict__ b, float* __restrict__ Z,
                                                            float* __restrict__ Y, int n, int K, int N, int silu)
{
    __shared__ __align__(16) MmaTiles S;
    const int row0 = blockIdx.y * kTile, col0 = blockIdx.x * kTile;
    float acc[2][4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kKs) {
        stage_tile([&](int r, int k) {
            const int gr = row0 + r, gk = k0 + k;
            return (gr < n && gk < K) ? X[(size_t)(rows ? rows[gr] : gr) * K + gk] : 0.0f;
        }, S.a_hi, S.a_lo);
        stage_tile([&](int r, int k) {
            const int gc = col0 + r, gk = k0 + k;
            return (gc < N && gk < K) ? __bfloat162float(W[(size_t)gc * K + gk]) : 0.0f;
        }, S.b_hi, nullptr);
        __syncthreads();
        mma_step(S, false, acc);
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int r, c;
                acc_coord(mt, nt, q, r, c);
                r += row0; c += col0;
                if (r >= n || c >= N) continue;
                const float z = acc[mt][nt][q] + b[c];
                if (Z) Z[(size_t)r * N + c] = z;
                Y[(size_t)r * N + c] = silu ? z / (1.0f + expf(-z)) : z;
            }
}

// dZ = dY * act'(Z)
__global__ void k_act_bwd(const float* __restrict__ Z, const float* __restrict__ dY, float* __restrict__ dZ,
                          size_t count, int silu)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (!silu) { dZ[i] = dY[i]; return; }
    const float z = Z[i], s = 1.0f / (1.0f + expf(-z));
    dZ[i] = dY[i] * (s * (1.0f + z * (1.0f - s)));
}

// dX[n][K] = dZ[n][N] W[N][K]
__global__ void __launch_bounds__(kMmaThreads) k_linear_dx(const float* __restrict__ dZ,
                                                           const __nv_bfloat16* __restrict__ W, float* __restrict__ dX,
                                                           int n, int K, int N)
{
    __shared__ __align__(16) MmaTiles S;
    const int row0 = blockIdx.y * kTile, col0 = blockIdx.x * kTile;
    float acc[2][4][4] = {};
    for (int j0 = 0; j0 < N; j0 += kKs) {
        stage_tile([&](int r, int j) {
            const int gr = row0 + r, gj = j0 + j;
            return (gr < n && gj < N) ? dZ[(size_t)gr * N + gj] : 0.0f;
        }, S.a_hi, S.a_lo);
        stage_tile([&](int r, int j) {
            const int gk = col0 + r, gj = j0 + j;
            return (gk < K && gj < N) ? __bfloat162float(W[(size_t)gj * K + gk]) : 0.0f;
        }, S.b_hi, nullptr);
        __syncthreads();
        mma_step(S, false, acc);
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int r, c;
                acc_coord(mt, nt, q, r, c);
                r += row0; c += col0;
                if (r < n && c < K) dX[(size_t)r * K + c] = acc[mt][nt][q];
            }
}

// Partial weight and bias gradients over the point range of split z = blockIdx.z:
// part[z][N*K + N] holds dW[N][K] = sum_p dZ[p][N] X[p][K] and db[N] = sum_p dZ[p][N] (the bias by the first
// column of blocks, one thread per output unit, points in order)
__global__ void __launch_bounds__(kMmaThreads) k_linear_dw(const float* __restrict__ dZ, const float* __restrict__ X,
                                                           const int* __restrict__ rows, float* __restrict__ part,
                                                           int n, int K, int N, int per_split)
{
    __shared__ __align__(16) MmaTiles S;
    const int n0 = blockIdx.y * kTile, k0 = blockIdx.x * kTile;
    const int p_begin = blockIdx.z * per_split;
    const int p_end = min(n, p_begin + per_split);
    float* out = part + (size_t)blockIdx.z * ((size_t)N * K + N);
    float acc[2][4][4] = {};
    for (int p0 = p_begin; p0 < p_end; p0 += kKs) {
        stage_tile([&](int r, int pp) {
            const int gp = p0 + pp;
            return (gp < p_end && n0 + r < N) ? dZ[(size_t)gp * N + n0 + r] : 0.0f;
        }, S.a_hi, S.a_lo);
        stage_tile([&](int r, int pp) {
            const int gp = p0 + pp;
            return (gp < p_end && k0 + r < K) ? X[(size_t)(rows ? rows[gp] : gp) * K + k0 + r] : 0.0f;
        }, S.b_hi, S.b_lo);
        __syncthreads();
        mma_step(S, true, acc);
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int r, c;
                acc_coord(mt, nt, q, r, c);
                r += n0; c += k0;
                if (r < N && c < K) out[(size_t)r * K + c] = acc[mt][nt][q];
            }
    if (blockIdx.x == 0 && threadIdx.x < kTile && n0 + (int)threadIdx.x < N) {
        const int r = n0 + threadIdx.x;
        float s = 0.0f;
        for (int p = p_begin; p < p_end; ++p) s += dZ[(size_t)p * N + r];
        out[(size_t)N * K + r] = s;
    }
}

// gW[N*K] and gb[N] = sum over the splits of the partials, in split order
__global__ void k_reduce_splits(const float* __restrict__ part, int splits, int N, int K, float* __restrict__ gW,
                                float* __restrict__ gb)
{
    const size_t total = (size_t)N * K + N;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * total + i];
    if (i < (size_t)N * K) gW[i] = s;
    else gb[i - (size_t)N * K] = s;
}

// mean squared error over n points x O outputs: per-block loss partials and dL/dY = 2 (Y - T) / (O n)
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, const int* __restrict__ rows,
                      float* __restrict__ dY, float* __restrict__ part, int n, int O)
{
    __shared__ float sm[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < O * n) {
        const int p = i / O, o = i - p * O;
        const float e = Y[i] - T[(size_t)(rows ? rows[p] : p) * O + o];
        dY[i] = 2.0f * e / ((float)O * (float)n);
        l = e * e;
    }
    sm[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// Adam (Kingma & Ba, 2015) on the FP32 master weights, refreshing their BF16 copies
__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, size_t count, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, size_t count)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) wb[i] = __float2bfloat16_rn(w[i]);
}

struct FMap {
    double cx, cy, ell, inv_span;   // x^ = asinh((x - cx) / ell) * inv_span
    float kn, ma, tw;               // normalised conditions
};

FMap make_fmap(const ugkwp_feature_map& f, double Kn, double Ma, double Tw)
{
    FMap m;
    m.cx = f.cx; m.cy = f.cy; m.ell = f.ell;
    m.inv_span = 1.0 / std::asinh(f.ext / f.ell);
    m.kn = (float)(2.0 * (std::log10(Kn) - std::log10(f.kn_lo)) / (std::log10(f.kn_hi) - std::log10(f.kn_lo)) - 1.0);
    m.ma = (float)(2.0 * (Ma - f.ma_lo) / (f.ma_hi - f.ma_lo) - 1.0);
    m.tw = (float)(2.0 * (Tw - f.tw_lo) / (f.tw_hi - f.tw_lo) - 1.0);
    return m;
}

bool fmap_valid(const ugkwp_feature_map* f)
{
    return f && f->ell > 0.0 && f->ext > 0.0 && f->kn_lo > 0.0 && f->kn_hi > f->kn_lo && f->ma_hi > f->ma_lo &&
           f->tw_hi > f->tw_lo;
}

// one feature row (F floats): sin/cos(2^k pi x^), sin/cos(2^k pi y^), k = 0..7, x^, y^, conditions, zeros.
// 2^k x^ is reduced exactly to r in [-1, 1] (same sine and cosine of pi r) before sinpi/cospi.
__device__ void feature_row(const FMap& m, double x, double y, float* out, int F)
{
    const double xh = asinh((x - m.cx) / m.ell) * m.inv_span;
    const double yh = asinh((y - m.cy) / m.ell) * m.inv_span;
    for (int k = 0; k < 8; ++k) {
        const double tx = ldexp(xh, k), ty = ldexp(yh, k);
        const double rx = tx - 2.0 * rint(0.5 * tx), ry = ty - 2.0 * rint(0.5 * ty);
        out[k] = (float)sinpi(rx);
        out[8 + k] = (float)cospi(rx);
        out[16 + k] = (float)sinpi(ry);
        out[24 + k] = (float)cospi(ry);
    }
    out[32] = (float)xh;
    out[33] = (float)yh;
    out[34] = m.kn;
    out[35] = m.ma;
    out[36] = m.tw;
    for (int k = kFeatUsed; k < F; ++k) out[k] = 0.0f;
}

__global__ void k_features(FMap m, const double* __restrict__ x, const double* __restrict__ y, int n, int F,
                           float* __restrict__ feat)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    feature_row(m, x[i], y ? y[i] : 0.0, feat + (size_t)i * F, F);
}

// training pair of cell c: features of its centroid and targets (log rho, u/U_inf, v/U_inf, log T) of W * scale
__global__ void k_dataset(FMap m, const double* __restrict__ xc, const double* __restrict__ yc,
                          const double* __restrict__ W, double scale, double U_inf, int C, int F,
                          float* __restrict__ feat, float* __restrict__ targ)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    feature_row(m, xc[c], yc ? yc[c] : 0.0, feat + (size_t)c * F, F);
    const double rho = W[4 * c] * scale, mx = W[4 * c + 1] * scale, my = W[4 * c + 2] * scale;
    const double E = W[4 * c + 3] * scale;
    const double u = mx / rho, v = my / rho;
    const double T = (E / rho - 0.5 * (u * u + v * v)) / (1.5 * ugk::kR);
    targ[4 * c] = (float)log(rho);
    targ[4 * c + 1] = (float)(u / U_inf);
    targ[4 * c + 2] = (float)(v / U_inf);
    targ[4 * c + 3] = (float)log(T);
}

// network outputs -> conservative W (clipped to rho in [1e-6, 1e6], T in [T_lo, T_hi], speed at most U_hi);
// the retained-particle tally is cleared, as for any new starting field
__global__ void k_apply_outputs(ugk::Dev d, const float* __restrict__ Y, int C, double U_inf, double T_lo,
                                double T_hi, double U_hi)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const double lr = fmin(fmax((double)Y[4 * c], -700.0), 700.0);
    const double lt = fmin(fmax((double)Y[4 * c + 3], -700.0), 700.0);
    const double rho = fmin(fmax(exp(lr), 1e-6), 1e6);
    double u = (double)Y[4 * c + 1] * U_inf, v = (double)Y[4 * c + 2] * U_inf;
    const double sp = sqrt(u * u + v * v);
    if (sp > U_hi) { u *= U_hi / sp; v *= U_hi / sp; }
    const double T = fmin(fmax(exp(lt), T_lo), T_hi);
    d.W[4 * c] = rho;
    d.W[4 * c + 1] = rho * u;
    d.W[4 * c + 2] = rho * v;
    d.W[4 * c + 3] = rho * (0.5 * (u * u + v * v) + 1.5 * ugk::kR * T);
    for (int k = 0; k < 5; ++k) d.wrt[5 * c + k] = 0;
}

__global__ void k_accumulate(const double* __restrict__ W, double* __restrict__ acc, int n, int reset)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[i] = reset ? W[i] : acc[i] + W[i];
}

unsigned nb(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct ugkwp_mlp {
    int F = 0, H = 0, L = 0, O = 0, cap = 0;
    std::vector<int> in, out;          // per layer (L + 1 layers)
    std::vector<size_t> woff, boff;    // offsets into the parameter vector
    size_t nparam = 0, part_len = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // FP32 master, gradient, Adam moments
    __nv_bfloat16* wb = nullptr;       // BF16 copy of every parameter (the biases' copies are unused)
    float *act = nullptr, *pre = nullptr, *dbuf = nullptr, *dpre = nullptr, *loss_part = nullptr, *part = nullptr;
    int64_t t = 0;
    cudaStream_t s = nullptr;
};

namespace {

ugkwp_status mlp_reserve(ugkwp_mlp* M, int cap)
{
    if (cap <= M->cap) return UGKWP_OK;
    const size_t per = (size_t)cap * M->H;
    cudaStreamSynchronize(M->s);
    cudaFree(M->act); cudaFree(M->pre); cudaFree(M->dbuf); cudaFree(M->dpre); cudaFree(M->loss_part);
    M->act = M->pre = M->dbuf = M->dpre = M->loss_part = nullptr;
    M->cap = 0;
    // activations of layers 1..L+1 (layer 0 is the caller's input) and pre-activations of layers 0..L, each
    // at a stride of cap x H floats; two gradient buffers that alternate between layers
    if (cudaMalloc(&M->act, sizeof(float) * per * (M->L + 1)) != cudaSuccess ||
        cudaMalloc(&M->pre, sizeof(float) * per * (M->L + 1)) != cudaSuccess ||
        cudaMalloc(&M->dbuf, sizeof(float) * per * 2) != cudaSuccess ||
        cudaMalloc(&M->dpre, sizeof(float) * per) != cudaSuccess ||
        cudaMalloc(&M->loss_part, sizeof(float) * (nb((size_t)M->O * cap, 256) + 1)) != cudaSuccess)
        return UGKWP_ENOMEM;
    M->cap = cap;
    return UGKWP_OK;
}

float* act_of(ugkwp_mlp* M, int layer) { return M->act + (size_t)(layer - 1) * M->cap * M->H; }   // layer >= 1
float* pre_of(ugkwp_mlp* M, int layer) { return M->pre + (size_t)layer * M->cap * M->H; }

// forward pass of n <= cap points; the output layer goes to Yout when given (else to act_of(L + 1))
void forward(ugkwp_mlp* M, const float* X, const int* rows, int n, float* Yout, bool keep)
{
    const float* x = X;
    for (int l = 0; l <= M->L; ++l) {
        const int K = M->in[l], N = M->out[l];
        float* y = (l == M->L && Yout) ? Yout : act_of(M, l + 1);
        dim3 grid(nb(N, kTile), nb(n, kTile));
        k_linear_fwd<<<grid, kMmaThreads, 0, M->s>>>(x, l == 0 ? rows : nullptr, M->wb + M->woff[l], M->p + M->boff[l],
                                            keep ? pre_of(M, l) : nullptr, y, n, K, N, l < M->L ? 1 : 0);
        x = y;
    }
}

}  // namespace

extern "C" {

ugkwp_status ugkwp_mlp_create(int32_t n_features, int32_t width, int32_t depth, int32_t n_out, const float* params,
                              void* stream, ugkwp_mlp** out)
{
    if (!out) return UGKWP_EINVAL;
    *out = nullptr;
    if (n_features < kFeatUsed || width <= 0 || depth <= 0 || n_out <= 0 || n_out > width) return UGKWP_EINVAL;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) return UGKWP_ECUDA;
    ugkwp_mlp* M = new (std::nothrow) ugkwp_mlp;
    if (!M) return UGKWP_ENOMEM;
    M->F = n_features; M->H = width > n_features ? width : n_features; M->L = depth; M->O = n_out;
    M->s = static_cast<cudaStream_t>(stream);
    for (int l = 0; l <= depth; ++l) {
        M->in.push_back(l == 0 ? n_features : width);
        M->out.push_back(l == depth ? n_out : width);
    }
    size_t maxlen = 0;
    for (int l = 0; l <= depth; ++l) {
        M->woff.push_back(M->nparam);
        M->nparam += (size_t)M->in[l] * M->out[l];
        const size_t len = (size_t)M->in[l] * M->out[l] + M->out[l];
        if (len > maxlen) maxlen = len;
    }
    for (int l = 0; l <= depth; ++l) {
        M->boff.push_back(M->nparam);
        M->nparam += (size_t)M->out[l];
    }
    M->part_len = maxlen;
    const size_t np = M->nparam;
    if (cudaMalloc(&M->p, 4 * np) != cudaSuccess || cudaMalloc(&M->g, 4 * np) != cudaSuccess ||
        cudaMalloc(&M->m, 4 * np) != cudaSuccess || cudaMalloc(&M->v, 4 * np) != cudaSuccess ||
        cudaMalloc(&M->wb, 2 * np) != cudaSuccess ||
        cudaMalloc(&M->part, sizeof(float) * maxlen * kMaxSplit) != cudaSuccess || mlp_reserve(M, 4096) != UGKWP_OK) {
        ugkwp_mlp_destroy(M);
        return UGKWP_ENOMEM;
    }
    if (params) cudaMemcpyAsync(M->p, params, 4 * np, cudaMemcpyHostToDevice, M->s);
    else cudaMemsetAsync(M->p, 0, 4 * np, M->s);
    cudaMemsetAsync(M->g, 0, 4 * np, M->s);
    cudaMemsetAsync(M->m, 0, 4 * np, M->s);
    cudaMemsetAsync(M->v, 0, 4 * np, M->s);
    k_to_bf16<<<nb(np, 256), 256, 0, M->s>>>(M->p, M->wb, np);
    if (cudaStreamSynchronize(M->s) != cudaSuccess) {
        ugkwp_mlp_destroy(M);
        return UGKWP_ECUDA;
    }
    *out = M;
    return UGKWP_OK;
}

void ugkwp_mlp_destroy(ugkwp_mlp* M)
{
    if (!M) return;
    cudaStreamSynchronize(M->s);
    cudaFree(M->p); cudaFree(M->g); cudaFree(M->m); cudaFree(M->v); cudaFree(M->wb); cudaFree(M->part);
    cudaFree(M->act); cudaFree(M->pre); cudaFree(M->dbuf); cudaFree(M->dpre); cudaFree(M->loss_part);
    delete M;
}

int64_t ugkwp_mlp_num_params(const ugkwp_mlp* M) { return M ? (int64_t)M->nparam : -1; }

ugkwp_status ugkwp_mlp_get_params(ugkwp_mlp* M, float* params, float* grad)
{
    if (!M || (!params && !grad)) return UGKWP_EINVAL;
    if (params && cudaMemcpyAsync(params, M->p, 4 * M->nparam, cudaMemcpyDeviceToHost, M->s) != cudaSuccess)
        return UGKWP_ECUDA;
    if (grad && cudaMemcpyAsync(grad, M->g, 4 * M->nparam, cudaMemcpyDeviceToHost, M->s) != cudaSuccess)
        return UGKWP_ECUDA;
    return cudaStreamSynchronize(M->s) == cudaSuccess ? UGKWP_OK : UGKWP_ECUDA;
}

ugkwp_status ugkwp_mlp_set_params(ugkwp_mlp* M, const float* params)
{
    if (!M || !params) return UGKWP_EINVAL;
    if (cudaMemcpyAsync(M->p, params, 4 * M->nparam, cudaMemcpyHostToDevice, M->s) != cudaSuccess) return UGKWP_ECUDA;
    cudaMemsetAsync(M->m, 0, 4 * M->nparam, M->s);
    cudaMemsetAsync(M->v, 0, 4 * M->nparam, M->s);
    M->t = 0;
    k_to_bf16<<<nb(M->nparam, 256), 256, 0, M->s>>>(M->p, M->wb, M->nparam);
    return cudaStreamSynchronize(M->s) == cudaSuccess ? UGKWP_OK : UGKWP_ECUDA;
}

ugkwp_status ugkwp_mlp_forward(ugkwp_mlp* M, const float* x_dev, int32_t n, float* y_dev)
{
    if (!M || n < 0 || (n > 0 && (!x_dev || !y_dev))) return UGKWP_EINVAL;
    for (int32_t p0 = 0; p0 < n; p0 += M->cap) {
        const int nn = n - p0 < M->cap ? n - p0 : M->cap;
        forward(M, x_dev + (size_t)p0 * M->F, nullptr, nn, y_dev + (size_t)p0 * M->O, false);
    }
    return cudaGetLastError() == cudaSuccess ? UGKWP_OK : UGKWP_ECUDA;
}

ugkwp_status ugkwp_mlp_grad(ugkwp_mlp* M, const float* x_dev, const float* t_dev, const int32_t* rows_dev, int32_t n,
                            float* loss)
{
    if (!M || !x_dev || !t_dev || n <= 0) return UGKWP_EINVAL;
    if (mlp_reserve(M, n) != UGKWP_OK) return UGKWP_ENOMEM;
    forward(M, x_dev, rows_dev, n, nullptr, true);
    const int L = M->L;
    const unsigned nblk_loss = nb((size_t)M->O * n, 256);
    float* dY = M->dbuf;
    k_mse<<<nblk_loss, 256, 0, M->s>>>(act_of(M, L + 1), t_dev, rows_dev, dY, M->loss_part, n, M->O);
    int splits = (n + kPointsPerSplit - 1) / kPointsPerSplit;
    if (splits > kMaxSplit) splits = kMaxSplit;
    const int per_split = (n + splits - 1) / splits;
    for (int l = L; l >= 0; --l) {
        const int K = M->in[l], N = M->out[l];
        const size_t cnt = (size_t)n * N;
        k_act_bwd<<<nb(cnt, 256), 256, 0, M->s>>>(pre_of(M, l), dY, M->dpre, cnt, l < L ? 1 : 0);
        const float* X = l == 0 ? x_dev : act_of(M, l);
        dim3 gw(nb(K, kTile), nb(N, kTile), splits);
        k_linear_dw<<<gw, kMmaThreads, 0, M->s>>>(M->dpre, X, l == 0 ? rows_dev : nullptr, M->part, n, K, N, per_split);
        k_reduce_splits<<<nb((size_t)N * K + N, 256), 256, 0, M->s>>>(M->part, splits, N, K, M->g + M->woff[l],
                                                                      M->g + M->boff[l]);
        if (l > 0) {
            float* dX = (dY == M->dbuf) ? M->dbuf + (size_t)M->cap * M->H : M->dbuf;
            dim3 gx(nb(K, kTile), nb(n, kTile));
            k_linear_dx<<<gx, kMmaThreads, 0, M->s>>>(M->dpre, M->wb + M->woff[l], dX, n, K, N);
            dY = dX;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return UGKWP_ECUDA;
    if (loss) {
        std::vector<float> part(nblk_loss);
        if (cudaMemcpyAsync(part.data(), M->loss_part, 4 * nblk_loss, cudaMemcpyDeviceToHost, M->s) != cudaSuccess ||
            cudaStreamSynchronize(M->s) != cudaSuccess)
            return UGKWP_ECUDA;
        double sum = 0.0;
        for (float x : part) sum += x;
        *loss = (float)(sum / ((double)M->O * n));
    }
    return UGKWP_OK;
}

ugkwp_status ugkwp_mlp_adam(ugkwp_mlp* M, float lr)
{
    if (!M || !(lr > 0.0f)) return UGKWP_EINVAL;
    M->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)M->t)), c2 = (float)(1.0 - std::pow(0.999, (double)M->t));
    k_adam<<<nb(M->nparam, 256), 256, 0, M->s>>>(M->p, M->wb, M->g, M->m, M->v, M->nparam, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? UGKWP_OK : UGKWP_ECUDA;
}

ugkwp_status ugkwp_mlp_features(const ugkwp_feature_map* fm, const double* x_dev, const double* y_dev, int32_t n,
                                double Kn, double Ma, double Tw, int32_t n_features, float* feat_dev, void* stream)
{
    if (!fmap_valid(fm) || n < 0 || n_features < kFeatUsed || !(Kn > 0.0) || (n > 0 && (!x_dev || !feat_dev)))
        return UGKWP_EINVAL;
    if (n == 0) return UGKWP_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_features<<<nb(n, 128), 128, 0, s>>>(make_fmap(*fm, Kn, Ma, Tw), x_dev, y_dev, n, n_features, feat_dev);
    return cudaGetLastError() == cudaSuccess ? UGKWP_OK : UGKWP_ECUDA;
}

ugkwp_status ugkwp_field_accumulate(ugkwp_ctx* h, double* acc_dev, int32_t reset)
{
    if (!h || !acc_dev) return UGKWP_EINVAL;
    ugk::Ctx& ctx = h->c;
    const int n = 4 * ctx.k.C;
    k_accumulate<<<nb(n, 256), 256, 0, ctx.stream>>>(ctx.d.W, acc_dev, n, reset ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? UGKWP_OK : UGKWP_ECUDA;
}

ugkwp_status ugkwp_mlp_dataset(ugkwp_ctx* h, const ugkwp_feature_map* fm, const double* W_dev, double scale,
                               int32_t n_features, float* feat_dev, float* targ_dev)
{
    if (!h || !fmap_valid(fm) || !feat_dev || !targ_dev || !(scale > 0.0) || n_features < kFeatUsed)
        return UGKWP_EINVAL;
    ugk::Ctx& ctx = h->c;
    const int C = ctx.k.C;
    k_dataset<<<nb(C, 128), 128, 0, ctx.stream>>>(make_fmap(*fm, ctx.Kn, ctx.Ma, ctx.k.Tw), ctx.d.xc,
                                                  ctx.k.dim == 2 ? ctx.d.yc : nullptr, W_dev ? W_dev : ctx.d.W,
                                                  W_dev ? scale : 1.0, ctx.k.U_inf, C, n_features, feat_dev, targ_dev);
    return cudaGetLastError() == cudaSuccess ? UGKWP_OK : UGKWP_ECUDA;
}

ugkwp_status ugkwp_warm_start(ugkwp_ctx* h, ugkwp_mlp* M, const ugkwp_feature_map* fm)
{
    if (!h || !M || !fmap_valid(fm) || M->O != 4) return UGKWP_EINVAL;
    ugk::Ctx& ctx = h->c;
    const int C = ctx.k.C;
    float *feat = nullptr, *y = nullptr;
    if (cudaMalloc(&feat, sizeof(float) * (size_t)C * M->F) != cudaSuccess ||
        cudaMalloc(&y, sizeof(float) * (size_t)C * 4) != cudaSuccess) {
        cudaFree(feat);
        return UGKWP_ENOMEM;
    }
    // the network runs on the context's stream
    cudaStream_t keep = M->s;
    cudaStreamSynchronize(keep);
    M->s = ctx.stream;
    k_features<<<nb(C, 128), 128, 0, ctx.stream>>>(make_fmap(*fm, ctx.Kn, ctx.Ma, ctx.k.Tw), ctx.d.xc,
                                                   ctx.k.dim == 2 ? ctx.d.yc : nullptr, C, M->F, feat);
    ugkwp_status st = ugkwp_mlp_forward(M, feat, C, y);
    M->s = keep;
    if (st == UGKWP_OK) {
        k_apply_outputs<<<nb(C, 128), 128, 0, ctx.stream>>>(ctx.d, y, C, ctx.k.U_inf, 2.0 * ctx.k.T_min,
                                                           0.5 * ctx.k.T_cap, 0.5 * ctx.k.U_cap);
        cudaMemsetAsync(ctx.d.counts, 0, sizeof(int), ctx.stream);   // no retained particles
        if (cudaStreamSynchronize(ctx.stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = UGKWP_ECUDA;
    }
    cudaFree(feat);
    cudaFree(y);
    return st;
}

}  // extern "C"
