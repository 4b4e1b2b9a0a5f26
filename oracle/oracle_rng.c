/* ORACLE (test infrastructure only; never linked into the product path).
 *
 * Philox4x32-10 counter-based generator, written from its published definition:
 * J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11. Ten rounds; each round multiplies counter words 0 and 2 by the two Philox multipliers, takes
 * the high and low halves of the 64-bit products, mixes them with counter words 1 and 3 and the key, and
 * permutes; the key is bumped by the two Weyl constants between rounds.
 *
 * The stream layout (which counter a draw uses) is the build's reading of a point the paper leaves open:
 * key = (seed_lo ^ case_id, seed_hi); counter = (pid_lo, pid_hi, step, draw).
 *
 * Uniforms in (0, 1), both exact in their format:
 *   float : ((w >> 9) + 0.5) * 2^-23
 *   double: (((hi:lo) >> 12) + 0.5) * 2^-52, with hi:lo the 64-bit word built from two outputs.
 */
#include "oracle_internal.h"

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n1 = lo1;
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    const uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

void or_draw(const or_ctx* cx, uint64_t pid, uint32_t draw, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)cx->step, draw};
    uint32_t key[2] = {(uint32_t)cx->seed ^ cx->case_id, (uint32_t)(cx->seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

float or_u01f(uint32_t w)
{
    return ((float)(w >> 9) + 0.5f) * 0x1p-23f;
}

double or_u01d(uint32_t lo, uint32_t hi)
{
    const uint64_t b = ((uint64_t)hi << 32) | (uint64_t)lo;
    return ((double)(b >> 12) + 0.5) * 0x1p-52;
}

/* j-th uniform of the draw group starting at counter word `base` (see the layout in the header) */
void or_uniforms_f(const or_ctx* cx, uint64_t pid, uint32_t base, int n, float* u)
{
    uint32_t w[4];
    or_draw(cx, pid, base, w);
    for (int j = 0; j < n; ++j) u[j] = or_u01f(w[j]);
}

void or_uniforms_d(const or_ctx* cx, uint64_t pid, uint32_t base, int n, double* u)
{
    uint32_t w[4];
    for (int j = 0; j < n; ++j) {
        if ((j & 1) == 0) or_draw(cx, pid, base + (uint32_t)(j >> 1), w);
        u[j] = or_u01d(w[2 * (j & 1)], w[2 * (j & 1) + 1]);
    }
}

/* exported for the known-answer test */
void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    or_philox4x32_10(ctr, key, out);
}
