/*
 * CPU oracle for the interference-sensitivity hot path — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests, the smoke check and the CPU-baseline leg of the benchmark may load
 * this library.  It is deliberately plain and slow: single-threaded loops, fp64
 * wherever floating point is not fixed by the definition, no blocking or fusion.
 * It shares no code, header or table with the CUDA library.
 *
 * Contents (each function cites what it follows):
 *   - SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the counter-based generator
 *     the stressor kernels draw their private seeds from.
 *   - Stressor checksums.  The paper's stressors (Sec. 3 "Pitfall 1/2" compute and
 *     copy kernels, Sec. 4.2 sleep kernel, Sec. 4.3 copy kernel, Sec. 4.4.1
 *     strided shared-memory copy) each hammer one resource; every kernel here
 *     folds the data it touched into a checksum so that skipped or duplicated
 *     work is visible.  The fold rules are this build's own definitions.
 *   - Victim kernels written from their textbook definitions in fp64: triad,
 *     GEMM, GEMV, layer normalisation, row softmax, 256-bin histogram.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* SplitMix64: output i of the generator started at state s0 is               */
/* mix(s0 + (i+1)*gamma), gamma = 0x9E3779B97F4A7C15.                        */
/* ------------------------------------------------------------------------- */
uint64_t or_splitmix64(uint64_t s0, uint64_t i) {
    uint64_t z = s0 + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint32_t rotl32(uint32_t x, unsigned r) {
    r &= 31u;
    return r ? (x << r) | (x >> (32u - r)) : x;
}

static uint32_t f32_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* ------------------------------------------------------------------------- */
/* L2 / HBM stream stressor (the paper's copy kernel, Sec. 3 Pitfall 2 and     */
/* Sec. 4.3).  The buffer of n int32 words is cut into chunks of chunk_elems   */
/* (a multiple of 4).  Active block k of A (planned) reads the chunks          */
/* c = k, k+A, k+2A, ... (m_k of them) in that order, cycling; its j-th chunk  */
/* read (j = 0..count-1) is chunk c_j = k + (j mod m_k)*A in pass              */
/* p_j = floor(j / m_k).  The kernel reads every word of every chunk and folds */
/* a part of it, by `fold`:                                                   */
/*   fold 0 (loads into registers): the first word of every 16-byte group,    */
/*          words 4i of the chunk, the words the register-load kernel loads;  */
/*   fold 1 (bulk copies into shared memory): quarter p_j mod 4 of the chunk  */
/*          (the chunk's four contiguous quarters), so four consecutive       */
/*          passes fold every word once.                                      */
/* The block's checksum is XOR_j rotl(F(c_j, p_j), p_j mod 32) where F is the */
/* XOR of the folded words.                                                   */
/* ------------------------------------------------------------------------- */
uint32_t or_stream_block_checksum(const uint32_t *buf, int64_t n_elems, int64_t chunk_elems,
                                  int64_t active_planned, int64_t k, int64_t count, int fold) {
    if (chunk_elems <= 0 || chunk_elems % 4 || active_planned <= 0 || k < 0 || count <= 0) return 0u;
    if (fold != 0 && fold != 1) return 0u;
    int64_t n_chunks = n_elems / chunk_elems;
    if (k >= n_chunks) return 0u;
    int64_t m_k = (n_chunks - k + active_planned - 1) / active_planned;
    int64_t quarter = chunk_elems / 4;
    uint32_t acc = 0u;
    for (int64_t j = 0; j < count; ++j) {
        int64_t c = k + (j % m_k) * active_planned;
        int64_t p = j / m_k;
        const uint32_t *w = buf + c * chunk_elems;
        uint32_t x = 0u;
        if (fold == 0) {
            for (int64_t e = 0; e < chunk_elems; e += 4) x ^= w[e];
        } else {
            int64_t q = p % 4;
            for (int64_t e = q * quarter; e < (q + 1) * quarter; ++e) x ^= w[e];
        }
        acc ^= rotl32(x, (unsigned)(p & 31));
    }
    return acc;
}

/* ------------------------------------------------------------------------- */
/* FP32 FMA stressor (the paper's compute kernel, Sec. 3 and Sec. 4.4.2: many  */
/* independent fp32 chains, ILP = chains per thread).  One multiplier and one  */
/* addend per launch, from outputs 0 and 1 of SplitMix64(seed<<32):            */
/*   a = 1 - 2^-12 - (u0>>53) * 2^-23          (exact in fp32, |a| < 1)        */
/*   b = ((u1>>40) - 2^23) * 2^-29                                             */
/* Chain j of thread t of active block k, g = (k*block + t)*ilp + j, starts at */
/*   x0 = ((u(g+2)>>40) - 2^23) * 2^-23                                        */
/* and iterates x <- fma(x, a, b) (one rounding), `steps` times per round.     */
/* round0_xor: XOR of the bits of every chain after round 0;                   */
/* final_xor: the same after `rounds` rounds.                                  */
/* ------------------------------------------------------------------------- */
void or_fma_block(uint64_t seed, int64_t k, int block, int ilp, int steps, int64_t rounds,
                  uint32_t *round0_xor, uint32_t *final_xor) {
    uint64_t s0 = seed << 32;
    float a = (float)(1.0 - ldexp(1.0, -12) - (double)(or_splitmix64(s0, 0) >> 53) * ldexp(1.0, -23));
    float b = (float)((double)((int64_t)(or_splitmix64(s0, 1) >> 40) - (1 << 23)) * ldexp(1.0, -29));
    uint32_t r0 = 0u, fin = 0u;
    for (int t = 0; t < block; ++t) {
        for (int j = 0; j < ilp; ++j) {
            uint64_t g = ((uint64_t)k * (uint64_t)block + (uint64_t)t) * (uint64_t)ilp + (uint64_t)j;
            float x = (float)((double)((int64_t)(or_splitmix64(s0, g + 2u) >> 40) - (1 << 23)) * ldexp(1.0, -23));
            for (int64_t r = 0; r < rounds; ++r) {
                for (int s = 0; s < steps; ++s) x = fmaf(x, a, b);
                if (r == 0) r0 ^= f32_bits(x);
            }
            fin ^= f32_bits(x);
        }
    }
    if (round0_xor) *round0_xor = r0;
    if (final_xor) *final_xor = fin;
}

/* ------------------------------------------------------------------------- */
/* FP64 stressor (the paper's compute kernel turned to fp64 multiplication,    */
/* Sec. 4.4.3, scenarios S1-S4 = ILP 1-4).  One multiplier per launch, from    */
/* output 0 of SplitMix64(seed<<32):                                           */
/*   a = 1 - (1 + (u0>>54)) * 2^-40            (exact in fp64, 0 < a < 1)      */
/* Chain j of thread t of active block k, g = (k*block + t)*ilp + j, starts at */
/*   x0 = 1 + (u(g+2)>>12) * 2^-52             (exact, in [1, 2))              */
/* and iterates x <- x * a (one IEEE rounding), `steps` times per round.  Each */
/* chain contributes the XOR of the two 32-bit halves of its bits.            */
/* round0_xor: XOR over chains after round 0; final_xor: after `rounds`.       */
/* ------------------------------------------------------------------------- */
static uint32_t f64_fold(double d) {
    uint64_t u;
    memcpy(&u, &d, sizeof u);
    return (uint32_t)(u ^ (u >> 32));
}

void or_fp64_block(uint64_t seed, int64_t k, int block, int ilp, int steps, int64_t rounds,
                   uint32_t *round0_xor, uint32_t *final_xor) {
    uint64_t s0 = seed << 32;
    double a = 1.0 - (double)(1u + (unsigned)(or_splitmix64(s0, 0) >> 54)) * ldexp(1.0, -40);
    uint32_t r0 = 0u, fin = 0u;
    for (int t = 0; t < block; ++t) {
        for (int j = 0; j < ilp; ++j) {
            uint64_t g = ((uint64_t)k * (uint64_t)block + (uint64_t)t) * (uint64_t)ilp + (uint64_t)j;
            double x = 1.0 + (double)(or_splitmix64(s0, g + 2u) >> 12) * ldexp(1.0, -52);
            for (int64_t r = 0; r < rounds; ++r) {
                for (int s = 0; s < steps; ++s) x = x * a;
                if (r == 0) r0 ^= f64_fold(x);
            }
            fin ^= f64_fold(x);
        }
    }
    if (round0_xor) *round0_xor = r0;
    if (final_xor) *final_xor = fin;
}

/* ------------------------------------------------------------------------- */
/* Shared-memory stressor (the paper's n-strided shared-memory copy, Sec.      */
/* 4.4.1).  Each warp owns a 4 KiB array of 1024 words, word q initialised to  */
/* low32(SplitMix64(seed<<32, (k*warps + w)*1024 + q)).  Every pass loads and  */
/* stores each word once; passes are numbered 0, 1, 2, ... over all rounds (a  */
/* round is `passes` passes) and the even ones apply the LCG                    */
/* w <- 1664525*w + 1013904223 (mod 2^32) while the odd ones copy the word.    */
/* The access order (and hence the bank-conflict degree) does not change the   */
/* result.  Returns the XOR of all words of the block.                         */
/* ------------------------------------------------------------------------- */
uint32_t or_smem_block(uint64_t seed, int64_t k, int warps, int64_t rounds, int passes) {
    uint64_t s0 = seed << 32;
    int64_t steps = (rounds * (int64_t)passes + 1) / 2; /* even pass indices */
    uint32_t acc = 0u;
    for (int w = 0; w < warps; ++w) {
        for (int q = 0; q < 1024; ++q) {
            uint32_t v = (uint32_t)or_splitmix64(s0, ((uint64_t)k * (uint64_t)warps + (uint64_t)w) * 1024u + (uint64_t)q);
            for (int64_t s = 0; s < steps; ++s) v = v * 1664525u + 1013904223u;
            acc ^= v;
        }
    }
    return acc;
}

/* ------------------------------------------------------------------------- */
/* BF16 tensor-pipe stressor.  Active block k holds A (128x64) and B (128x64,  */
/* K-major) with small-integer entries                                        */
/*   A[m][c] = ((SplitMix64(seed<<32, k*16384 + m*64 + c) >> 32) mod 5) - 2   */
/*   B[n][c] = same at k*16384 + 8192 + n*64 + c                               */
/* A round accumulates `group` products P = A B^T into a zeroed fp32 tile, so  */
/* the tile holds group*P exactly (|group*P| <= 2^24).  Returns the XOR of the */
/* fp32 bit patterns of the 128x128 tile.                                     */
/* ------------------------------------------------------------------------- */
uint32_t or_tensor_block(uint64_t seed, int64_t k, int group) {
    uint64_t s0 = seed << 32;
    static int A[128][64], B[128][64];
    for (int m = 0; m < 128; ++m)
        for (int c = 0; c < 64; ++c) {
            A[m][c] = (int)((or_splitmix64(s0, (uint64_t)k * 16384u + (uint64_t)(m * 64 + c)) >> 32) % 5u) - 2;
            B[m][c] = (int)((or_splitmix64(s0, (uint64_t)k * 16384u + 8192u + (uint64_t)(m * 64 + c)) >> 32) % 5u) - 2;
        }
    uint32_t acc = 0u;
    for (int m = 0; m < 128; ++m)
        for (int n = 0; n < 128; ++n) {
            int64_t p = 0;
            for (int c = 0; c < 64; ++c) p += (int64_t)A[m][c] * B[n][c];
            acc ^= f32_bits((float)((double)p * (double)group));
        }
    return acc;
}

/* ------------------------------------------------------------------------- */
/* Block-scheduler stressor (Sec. 4.2: many short blocks).  Block q of the     */
/* run (q = launch*blocks_per_launch + blockIdx) contributes                  */
/* y = LCG^lcg_steps(low32(q) ^ low32(seed)).  Returns the XOR over q < total. */
/* ------------------------------------------------------------------------- */
uint32_t or_sched_checksum(uint64_t seed, int64_t total_blocks, int lcg_steps) {
    uint32_t acc = 0u;
    for (int64_t q = 0; q < total_blocks; ++q) {
        uint32_t y = (uint32_t)q ^ (uint32_t)seed;
        for (int s = 0; s < lcg_steps; ++s) y = y * 1664525u + 1013904223u;
        acc ^= y;
    }
    return acc;
}

/* Plain affine composition of the LCG used above, n steps: v -> A v + C.     */
void or_lcg_power(int64_t n, uint32_t *A, uint32_t *C) {
    uint32_t a = 1u, c = 0u;
    for (int64_t s = 0; s < n; ++s) {
        a = a * 1664525u;
        c = c * 1664525u + 1013904223u;
    }
    *A = a;
    *C = c;
}

/* ------------------------------------------------------------------------- */
/* Victims (textbook definitions, fp64).                                      */
/* ------------------------------------------------------------------------- */

/* STREAM triad: a[i] = b[i] + s*c[i]. */
void or_triad(const float *b, const float *c, float s, int64_t n, double *a) {
    for (int64_t i = 0; i < n; ++i) a[i] = (double)b[i] + (double)s * (double)c[i];
}

/* Layer normalisation of selected rows (no affine, biased variance):          */
/* y = (x - mean) / sqrt(var + eps), mean and var by two passes in fp64.       */
void or_layernorm_rows(const float *x, int64_t cols, double eps, const int64_t *rows, int64_t n_rows,
                       double *y) {
    for (int64_t r = 0; r < n_rows; ++r) {
        const float *xr = x + rows[r] * cols;
        double mean = 0.0, var = 0.0;
        for (int64_t j = 0; j < cols; ++j) mean += (double)xr[j];
        mean /= (double)cols;
        for (int64_t j = 0; j < cols; ++j) {
            double d = (double)xr[j] - mean;
            var += d * d;
        }
        var /= (double)cols;
        double inv = 1.0 / sqrt(var + eps);
        for (int64_t j = 0; j < cols; ++j) y[r * cols + j] = ((double)xr[j] - mean) * inv;
    }
}

/* Row softmax of selected rows: y_j = exp(x_j - max) / sum_i exp(x_i - max). */
void or_softmax_rows(const float *x, int64_t cols, const int64_t *rows, int64_t n_rows, double *y) {
    for (int64_t r = 0; r < n_rows; ++r) {
        const float *xr = x + rows[r] * cols;
        double mx = -INFINITY, sum = 0.0;
        for (int64_t j = 0; j < cols; ++j)
            if ((double)xr[j] > mx) mx = (double)xr[j];
        for (int64_t j = 0; j < cols; ++j) sum += exp((double)xr[j] - mx);
        for (int64_t j = 0; j < cols; ++j) y[r * cols + j] = exp((double)xr[j] - mx) / sum;
    }
}

static double bf16_to_f64(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* GEMV of selected rows: y[r] = sum_c A[r][c] * x[c]; A row-major bf16.      */
void or_gemv_rows(const uint16_t *A, const uint16_t *x, int64_t cols, const int64_t *rows, int64_t n_rows,
                  double *y) {
    for (int64_t r = 0; r < n_rows; ++r) {
        double acc = 0.0;
        const uint16_t *ar = A + rows[r] * cols;
        for (int64_t c = 0; c < cols; ++c) acc += bf16_to_f64(ar[c]) * bf16_to_f64(x[c]);
        y[r] = acc;
    }
}

/* GEMM entries: C[i][j] = sum_k A[i][k] * B[j][k]; A is M x K row-major and B */
/* is N x K row-major (B stored K-major), both bf16.  ij holds (i, j) pairs.   */
void or_gemm_entries(const uint16_t *A, const uint16_t *B, int64_t K, const int64_t *ij, int64_t n,
                     double *c) {
    for (int64_t e = 0; e < n; ++e) {
        const uint16_t *a = A + ij[2 * e] * K;
        const uint16_t *b = B + ij[2 * e + 1] * K;
        double acc = 0.0;
        for (int64_t k = 0; k < K; ++k) acc += bf16_to_f64(a[k]) * bf16_to_f64(b[k]);
        c[e] = acc;
    }
}

/* 256-bin histogram of key & 255. */
void or_histogram(const int32_t *keys, int64_t n, uint64_t *bins) {
    for (int b = 0; b < 256; ++b) bins[b] = 0u;
    for (int64_t i = 0; i < n; ++i) bins[(uint32_t)keys[i] & 255u] += 1u;
}
