// Resource stressors (Sec. 3 compute/copy kernels, Sec. 4.2 block-scheduler kernel,
// Sec. 4.3 copy kernel over L2- and HBM-sized buffers, Sec. 4.4.1 strided
// shared-memory copy, Sec. 4.4.2 compute kernel with an ILP knob).
//
// Persistent kinds share one skeleton:
//   entry   thread 0 claims a slot on its SM (mask + blocks_per_sm); blocks that
//           fail exit at once.  The claim order gives the active index k.
//   rounds  thread 0 decides once per round (stop flag, max_rounds, deadline,
//           duty-cycle off phase) and broadcasts through shared memory.
//   exit    per-block log: %globaltimer entry/exit, rounds, work, checksums, %smid.
// Every wait (duty-cycle sleep, residency wait) is bounded by the block's deadline
// and an iteration cap; on expiry the block records IFR_ERR_TIMEOUT and returns.
#include <stdio.h>
#include <string.h>
#include <time.h>

#include <mutex>

#include <cuda_bf16.h>

#include "ifr_internal.cuh"
#include "ifr_tcgen05.cuh"

namespace {

constexpr int kStreamChunksPerRound = 8;  // L2/HBM: chunks per round (8 x 4 loads in flight per thread)
// FMA: steps per chain per round = kFmaWork / ILP (16384 FMAs per thread per round)
constexpr int kFmaWork = 16384;
// FP64: steps per chain per round = kFp64Work / ILP (1024 multiplies per thread per round)
constexpr int kFp64Work = 1024;
// SMEM: passes over the warp array per round = max(1, 32 / WAYS), so that every
// conflict degree spends the same 2048 wavefronts per warp per round (32 ld/st
// pairs per lane per pass, WAYS wavefronts each) and the once-per-round stop /
// deadline check costs the same small share of every variant
constexpr int kSmemPassesCF = 32;
constexpr int kSchedLcgSteps = 16;        // SCHED: LCG steps per block result
constexpr uint32_t kMaxSpin = 1u << 22;   // iteration cap of every sleep loop

// SplitMix64 (Steele, Lea, Flood 2014) on the host: output i of the stream at s0.
uint64_t host_splitmix64(uint64_t s0, uint64_t i) {
    uint64_t z = s0 + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct BlockCtl {
    int k;            // active index, -1 = not active
    uint64_t t0;      // entry time
    uint64_t deadline;
    int status;
};

// Duty-cycle state of a block (thread 0 only): start of the next period, the
// active time the block may still spend (each period adds its share, each round
// takes its duration, so what a round overran or left unused carries over), and
// the start of the running round.  It lives in shared memory, so the round loops
// keep their registers.
struct DutyState {
    uint64_t next;
    int64_t budget;
    uint64_t t_rs;
};

__device__ __forceinline__ bool sm_allowed(const StressParams &p, uint32_t sm) {
    return sm < IFR_MAX_SMS && ((p.mask[sm >> 5] >> (sm & 31)) & 1u);
}

__global__ void stress_reset_kernel(DevStress *st) {
    for (int i = threadIdx.x; i < IFR_MAX_SMS; i += blockDim.x) st->sm_claim[i] = 0u;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        st->sched_xor[i] = 0u;
        st->sched_cnt[i] = 0u;
    }
    if (threadIdx.x == 0) {
        st->stop = 0u;
        st->arrived = 0u;
        st->active = 0u;
        st->status = 0;
        st->t_origin = 0ull;
        st->t_first_start = ~0ull;
        st->t_last_end = 0ull;
        st->t_stop_seen = ~0ull;
    }
}

// Thread 0 only.  Claims an SM slot; returns the active index or -1.
__device__ int claim_slot(DevStress *st, const StressParams &p, uint32_t sm) {
    int k = -1;
    if (sm_allowed(p, sm)) {
        uint32_t slot = atomicAdd(&st->sm_claim[sm], 1u);
        if (slot < (uint32_t)p.bps) {
            int kk = (int)atomicAdd(&st->active, 1u);
            if (kk < p.planned) k = kk;
        }
    }
    __threadfence();
    atomicAdd(&st->arrived, 1u);
    if (k < 0 && p.planned > 0) {
        // A surplus block stays resident (bounded) until every planned slot is
        // claimed: the grid equals the GPU's block capacity, so while nobody
        // leaves, each allowed SM holds enough blocks to fill its slots.
        const uint64_t t_end = ifr_gtimer() + 200000ull;
        uint32_t it = 0;
        while (ifr_ld_volatile(&st->active) < (uint32_t)p.planned && ifr_gtimer() < t_end && ++it < kMaxSpin)
            __nanosleep(256);
    }
    return k;
}

// Sleep part of the way toward a %globaltimer target `left` ns away.  __nanosleep's
// duration is approximate (the PTX ISA allows anything up to twice the request), so
// a request of the whole distance can wake a block microseconds late.  Half the
// distance (at most 20 us) never passes the target; the last microsecond is polled.
__device__ __forceinline__ void sleep_toward(uint64_t left) {
    if (left > 1000u) __nanosleep((unsigned)(left > 40000u ? 20000u : left / 2));
}

// Thread 0 only: should the block run round `round`?  Sleeps through the
// off phase of the duty cycle.
__device__ int round_decision(DevStress *st, const StressParams &p, int64_t round, BlockCtl &c) {
    __shared__ DutyState s_duty;
    if (p.max_rounds > 0 && round >= p.max_rounds) return 0;
    if (ifr_ld_volatile(&st->stop)) return 0;
    uint64_t now = ifr_gtimer();
    if (now >= c.deadline) {
        c.status = IFR_ERR_TIMEOUT;
        return 0;
    }
    if (p.progress) {
        // head-of-line watch: a victim block must have entered or left within hol_ns
        uint64_t last = *(const volatile uint64_t *)p.progress;
        if (last < c.t0) last = c.t0;
        if (now > last + p.hol_ns) {
            c.status = IFR_ERR_HOL;
            return 0;
        }
    }
    if (p.duty_on_ns) {
        // Duty cycle D over period P: the periods are aligned on %globaltimer, so every
        // block of the launch is active in the same on-phase (the resource sees the full
        // stressor for D*P, then nothing).  A round that has started runs to its end;
        // each period adds D*P to the block's budget and each round takes its duration,
        // so the active fraction averages to D whatever the round length (the budget is
        // bounded by one period either way).  The first period adds only the share of
        // D*P for the part of it left after the block starts.
        DutyState &d = s_duty;
        const uint32_t per = p.period_ns;
        const int64_t on = p.duty_on_ns, lim = per;
        if (round == 0) {
            d.next = now - now % per + per;
            d.budget = (int64_t)((float)on * (float)(d.next - now) * p.duty_inv_period);
            d.t_rs = 0;
        }
        if (d.t_rs) {
            d.budget -= (int64_t)(now - d.t_rs);
            d.t_rs = 0;
        }
        uint32_t it = 0;
        for (;;) {
            if (now >= d.next) {
                d.budget += on;
                d.next += per;
                if (d.budget > lim) d.budget = lim;
                if (d.budget < -lim) d.budget = -lim;
                if (++it > kMaxSpin) return 0;
                continue;
            }
            if (d.budget > 0) break;
            while (now < d.next) {
                if (now >= c.deadline) {
                    c.status = IFR_ERR_TIMEOUT;
                    return 0;
                }
                if (ifr_ld_volatile(&st->stop) || ++it > kMaxSpin) return 0;
                sleep_toward(d.next - now);
                now = ifr_gtimer();
            }
        }
        d.t_rs = now;
    }
    return 1;
}

__device__ void write_log(const StressParams &p, DevStress *st, const BlockCtl &c, int64_t rounds, uint64_t work,
                          uint32_t cs, uint32_t cs2) {
    ifr_block_log L;
    L.t_start_ns = c.t0;
    L.t_end_ns = ifr_gtimer();
    L.rounds = (uint64_t)rounds;
    L.work = work;
    L.checksum = cs;
    L.checksum2 = cs2;
    L.smid = ifr_smid();
    L.index = c.k;
    L.status = c.status;
    L.reserved = 0u;
    p.logs[c.k] = L;
    if (c.status != 0) atomicCAS(&st->status, 0, c.status);
}

// Common entry; returns false (whole block) when the block is not active.
__device__ __forceinline__ bool block_enter(DevStress *st, const StressParams &p, BlockCtl &c, int *s_k,
                                            uint64_t *s_t0) {
    if (threadIdx.x == 0) {
        uint64_t t = ifr_gtimer();
        *s_k = claim_slot(st, p, ifr_smid());
        *s_t0 = t;
    }
    __syncthreads();
    c.k = *s_k;
    c.t0 = *s_t0;
    c.deadline = c.t0 + p.deadline_ns;
    c.status = 0;
    return c.k >= 0;
}

// ------------------------------------------------------------------ L2 / HBM
// The first 4-byte word of the 16-byte group at p.
__device__ __forceinline__ uint32_t ld_stream_word(const int4 *p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Every chunk is read whole: each thread loads the first word of each of its four
// 16-byte groups.  The 32 lanes of a warp load words 16 bytes apart, 512 contiguous
// bytes, so every 32-byte sector of the chunk is requested and moves whole from HBM
// into L2 and from L2 into the SM (memory moves in sectors, not words); a word load
// takes one register where a 16-byte load takes four.  Every loaded word enters the
// fold (a load whose result nothing used would be dropped by the compiler).
// BLK: the block size at compile time (128, 256 or 512), so the four loads of
// a chunk address it with immediate offsets; 0 reads blockDim.x at run time and
// takes every round chunk by chunk.  With BLK, a round whose R chunks need no wrap
// to the block's first chunk (all but about one round in n_chunks / (A R)) issues its
// R x 4 loads from one pointer with fixed offsets and folds them under one rotation;
// a round that wraps takes the chunks one by one.  The walk keeps one offset from the
// block's first chunk, compared with the offset of its last (the host refuses sets of
// more than 2^30 chunks, so counts fit 32 bits).  Every instantiation compiles to 32
// registers, the budget that leaves room for a victim block beside a full-intensity
// stressor.  (A launch bound asking for 2048 threads per SM gives the same count but
// measured 5 % less L2 bandwidth: the compiler keeps fewer loads in flight.)  Measured against the same word loads
// taken chunk by chunk with run-time offsets, in one process: 7.1 against 6.0-6.3
// TB/s from HBM and 17.1-18.7 against 16.0-18.0 TB/s from L2 over four block shapes.
template <int BLK>
__global__ void __launch_bounds__(BLK ? BLK : 1024)
    stream_stress_kernel(DevStress *st, StressParams p) {
    __shared__ int s_k;
    __shared__ uint64_t s_t0;
    __shared__ int s_go[2];
    __shared__ uint32_t s_red[32];
    BlockCtl c;
    if (!block_enter(st, p, c, &s_k, &s_t0)) return;
    constexpr int R = kStreamChunksPerRound;
    const int B = BLK ? BLK : (int)blockDim.x;
    const int A = (int)p.planned;
    const int k = c.k;
    const int n_chunks = (int)p.n_chunks;
    const bool has_work = k < n_chunks;
    // the thread's first int4 of the block's first chunk (k); the block's chunks k,
    // k + A, ..., k + (m - 1) A lie `stride` int4 apart, and `off` (int4 from `first`)
    // walks them, back to 0 after the last one (off_last)
    const int4 *const first = p.buf + (int64_t)k * (4 * B) + threadIdx.x;
    const int64_t stride = (int64_t)A * (4 * B);
    const int m = has_work ? (n_chunks - k + A - 1) / A : 1;
    const int64_t off_last = (int64_t)(m - 1) * stride;
    int64_t off = 0, done = 0;
    uint32_t pass = 0u, acc = 0u;
    int64_t round = 0;
    for (;; ++round) {
        if (threadIdx.x == 0) s_go[round & 1] = has_work ? round_decision(st, p, round, c) : 0;
        __syncthreads();
        if (!s_go[round & 1]) break;
        uint32_t v[R][4];
        if (BLK && off + (R - 1) * stride <= off_last) {
            // R chunks in a row of the cycle, one pass
            const int4 *src = first + off;
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int u = 0; u < 4; ++u) v[r][u] = ld_stream_word(src + r * stride + u * B);
            uint32_t x = 0u;
#pragma unroll
            for (int r = 0; r < R; ++r) x ^= v[r][0] ^ v[r][1] ^ v[r][2] ^ v[r][3];
            acc ^= ifr_rotl(x, pass);
            off += (R - 1) * stride;
            if (off == off_last) {
                off = 0;
                ++pass;
            } else {
                off += stride;
            }
        } else if (BLK) {
            uint32_t ps[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int4 *src = first + off;
#pragma unroll
                for (int u = 0; u < 4; ++u) v[r][u] = ld_stream_word(src + u * B);
                ps[r] = pass;
                if (off == off_last) {
                    off = 0;
                    ++pass;
                } else {
                    off += stride;
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) acc ^= ifr_rotl(v[r][0] ^ v[r][1] ^ v[r][2] ^ v[r][3], ps[r]);
        } else {
            // run-time block size: each chunk folded after its own loads (fewer live
            // registers where the offsets are not immediates)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int4 *q = first + off;
                uint32_t x = 0u;
#pragma unroll
                for (int u = 0; u < 4; ++u, q += B) x ^= ld_stream_word(q);
                acc ^= ifr_rotl(x, pass);
                if (off == off_last) {
                    off = 0;
                    ++pass;
                } else {
                    off += stride;
                }
            }
        }
        done += R;
    }
    uint32_t cs = ifr_block_xor(acc, s_red);
    if (threadIdx.x == 0) write_log(p, st, c, round, (uint64_t)done, cs, 0u);
}

// The stream kernel for a block size, and its launch.
const void *stream_fn(int block) {
    switch (block) {
        case 128: return (const void *)stream_stress_kernel<128>;
        case 256: return (const void *)stream_stress_kernel<256>;
        case 512: return (const void *)stream_stress_kernel<512>;
        default: return (const void *)stream_stress_kernel<0>;
    }
}
void launch_stream(int grid, int block, cudaStream_t stream, DevStress *st, const StressParams &p) {
    switch (block) {
        case 128: stream_stress_kernel<128><<<grid, block, 0, stream>>>(st, p); break;
        case 256: stream_stress_kernel<256><<<grid, block, 0, stream>>>(st, p); break;
        case 512: stream_stress_kernel<512><<<grid, block, 0, stream>>>(st, p); break;
        default: stream_stress_kernel<0><<<grid, block, 0, stream>>>(st, p);
    }
}

// The same stressor with TMA staging: a ring of p.ring stages of one chunk each in
// shared memory.  Thread 0 keeps the ring filled with whole-chunk bulk copies
// (cp.async.bulk, global -> this CTA's shared memory, completion counted in bytes
// on the stage's mbarrier) and waits for each chunk to land; one block barrier per
// chunk then lets every thread fold its 16 bytes of the chunk's quarter (pass & 3)
// from shared memory and tells thread 0 that the previous chunk's stage is free to
// refill.  The load/store unit carries only those 16-byte shared-memory reads and
// only thread 0 polls.  Every wait is bounded; a block drains the copies it issued
// before it exits, so no copy lands in shared memory that another block may own.
constexpr int kTmaMaxStages = 6;

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
        : "memory");
}

__global__ void __launch_bounds__(1024) stream_stress_tma_kernel(DevStress *st, StressParams p) {
    extern __shared__ __align__(128) uint8_t s_ring[];
    __shared__ __align__(8) uint64_t s_full[kTmaMaxStages];
    __shared__ int s_k;
    __shared__ uint64_t s_t0;
    __shared__ int s_go[2];
    __shared__ int s_fail;
    __shared__ uint32_t s_red[32];
    BlockCtl c;
    if (!block_enter(st, p, c, &s_k, &s_t0)) return;
    const int64_t A = p.planned, k = c.k;
    const int S = p.ring;
    const uint32_t chunk_bytes = blockDim.x * 64u;
    const bool has_work = k < p.n_chunks;
    const uint64_t wait_limit = c.deadline + 100000000ull;  // a copy gets 100 ms past the deadline
    int64_t ipos = k, issued = 0, landed = 0;  // thread 0: next chunk to copy, copies issued, seen landed
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) tc::mbar_init(&s_full[s], 1);
        s_fail = 0;
        tc::fence_mbar_init();
        if (has_work) {
            for (int s = 0; s < S; ++s, ++issued) {
                tc::mbar_arrive_expect_tx(&s_full[s], chunk_bytes);
                bulk_copy_g2s(s_ring + (size_t)s * chunk_bytes, (const uint8_t *)p.buf + ipos * chunk_bytes,
                              chunk_bytes, &s_full[s]);
                ipos += A;
                if (ipos >= p.n_chunks) ipos = k;
            }
        }
    }
    __syncthreads();
    int64_t cpos = k, pass = 0, done = 0, j = 0;
    int s = 0, sp = S - 1;  // stage of chunk j and of chunk j - 1
    uint32_t par = 0u;      // phase parity of chunk j's stage
    uint32_t acc = 0u;
    int64_t round = 0;
    for (;; ++round) {
        if (threadIdx.x == 0) s_go[round & 1] = (has_work && !s_fail) ? round_decision(st, p, round, c) : 0;
        __syncthreads();
        if (!s_go[round & 1]) break;
#pragma unroll 1
        for (int r = 0; r < kStreamChunksPerRound; ++r, ++j) {
            if (threadIdx.x == 0 && !s_fail) {
                if (tc::mbar_wait(&s_full[s], par, wait_limit))
                    landed = j + 1;
                else
                    s_fail = 1;
            }
            // chunk j has landed, and every thread has finished with chunk j - 1
            __syncthreads();
            if (threadIdx.x == 0 && j > 0 && !s_fail) {
                // refill the stage of chunk j - 1 with the chunk S reads ahead of it
                tc::mbar_arrive_expect_tx(&s_full[sp], chunk_bytes);
                bulk_copy_g2s(s_ring + (size_t)sp * chunk_bytes, (const uint8_t *)p.buf + ipos * chunk_bytes,
                              chunk_bytes, &s_full[sp]);
                ipos += A;
                if (ipos >= p.n_chunks) ipos = k;
                ++issued;
            }
            if (!s_fail) {
                const int4 *q = (const int4 *)(s_ring + (size_t)s * chunk_bytes) + (int)(pass & 3) * (int)blockDim.x +
                                (int)threadIdx.x;
                int4 v;
                asm volatile("ld.shared.v4.s32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                             : "r"(tc::smem_u32(q))
                             : "memory");
                acc ^= ifr_rotl((uint32_t)(v.x ^ v.y ^ v.z ^ v.w), (uint32_t)pass);
            }
            cpos += A;
            if (cpos >= p.n_chunks) {
                cpos = k;
                ++pass;
            }
            sp = s;
            if (++s == S) {
                s = 0;
                par ^= 1u;
            }
        }
        done += kStreamChunksPerRound;
    }
    // drain: every copy this block issued has landed before it exits
    if (threadIdx.x == 0) {
        for (int64_t q = landed; q < issued; ++q)
            if (!tc::mbar_wait(&s_full[q % S], (uint32_t)(q / S) & 1u, wait_limit)) s_fail = 1;
        if (s_fail && c.status == 0) c.status = IFR_ERR_TIMEOUT;
    }
    uint32_t cs = ifr_block_xor(acc, s_red);
    if (threadIdx.x == 0) write_log(p, st, c, round, (uint64_t)done, cs, 0u);
}

// ------------------------------------------------------------------ FP32 FMA
template <int ILP>
__global__ void __launch_bounds__(1024) fma_stress_kernel(DevStress *st, StressParams p) {
    __shared__ int s_k;
    __shared__ uint64_t s_t0;
    __shared__ int s_go[2];
    __shared__ uint32_t s_red[32];
    BlockCtl c;
    if (!block_enter(st, p, c, &s_k, &s_t0)) return;
    const uint64_t s0 = p.seed << 32;
    // the multiplier and addend are launch-wide kernel parameters, so each FFMA
    // reads a single register operand (x) and never stalls on register banks
    const float a = p.fma_a, b = p.fma_b;
    float x[ILP];
#pragma unroll
    for (int j = 0; j < ILP; ++j) {
        const uint64_t g = ((uint64_t)c.k * blockDim.x + threadIdx.x) * ILP + j;
        const uint64_t u0 = ifr_splitmix64(s0, g + 2ull);
        x[j] = (float)((int)(u0 >> 40) - (1 << 23)) * 0x1p-23f;
    }
    uint32_t r0 = 0u;
    int64_t round = 0;
    for (;; ++round) {
        if (threadIdx.x == 0) s_go[round & 1] = round_decision(st, p, round, c);
        __syncthreads();
        if (!s_go[round & 1]) break;
#pragma unroll 16
        for (int s = 0; s < kFmaWork / ILP; ++s) {
#pragma unroll
            for (int j = 0; j < ILP; ++j) x[j] = __fmaf_rn(x[j], a, b);
        }
        if (round == 0) {
#pragma unroll
            for (int j = 0; j < ILP; ++j) r0 ^= __float_as_uint(x[j]);
        }
    }
    uint32_t fin = 0u;
#pragma unroll
    for (int j = 0; j < ILP; ++j) fin ^= __float_as_uint(x[j]);
    uint32_t cs = ifr_block_xor(r0, s_red);
    uint32_t cs2 = ifr_block_xor(fin, s_red);
    if (threadIdx.x == 0) write_log(p, st, c, round, (uint64_t)round * (kFmaWork / ILP), cs, cs2);
}

// ------------------------------------------------------------------ FP64 multiply
// The compute kernel of Sec. 4.4.3 on fp64 multiplication (__dmul_rn): ILP
// independent chains x <- x * a per thread, one launch-wide multiplier just below 1.
template <int ILP>
__global__ void __launch_bounds__(1024, 1) fp64_stress_kernel(DevStress *st, StressParams p) {
    __shared__ int s_k;
    __shared__ uint64_t s_t0;
    __shared__ int s_go[2];
    __shared__ uint32_t s_red[32];
    BlockCtl c;
    if (!block_enter(st, p, c, &s_k, &s_t0)) return;
    const uint64_t s0 = p.seed << 32;
    const double a = p.fp64_a;
    double x[ILP];
#pragma unroll
    for (int j = 0; j < ILP; ++j) {
        const uint64_t g = ((uint64_t)c.k * blockDim.x + threadIdx.x) * ILP + j;
        x[j] = 1.0 + (double)(ifr_splitmix64(s0, g + 2ull) >> 12) * 0x1p-52;
    }
    uint32_t r0 = 0u;
    int64_t round = 0;
    for (;; ++round) {
        if (threadIdx.x == 0) s_go[round & 1] = round_decision(st, p, round, c);
        __syncthreads();
        if (!s_go[round & 1]) break;
#pragma unroll 8
        for (int s = 0; s < kFp64Work / ILP; ++s) {
#pragma unroll
            for (int j = 0; j < ILP; ++j) x[j] = __dmul_rn(x[j], a);
        }
        if (round == 0) {
#pragma unroll
            for (int j = 0; j < ILP; ++j) {
                const uint64_t u = (uint64_t)__double_as_longlong(x[j]);
                r0 ^= (uint32_t)(u ^ (u >> 32));
            }
        }
    }
    uint32_t fin = 0u;
#pragma unroll
    for (int j = 0; j < ILP; ++j) {
        const uint64_t u = (uint64_t)__double_as_longlong(x[j]);
        fin ^= (uint32_t)(u ^ (u >> 32));
    }
    uint32_t cs = ifr_block_xor(r0, s_red);
    uint32_t cs2 = ifr_block_xor(fin, s_red);
    if (threadIdx.x == 0) write_log(p, st, c, round, (uint64_t)round * (kFp64Work / ILP), cs, cs2);
}

// ------------------------------------------------------------------ sleep
// The sleep kernel of Sec. 4.2: each active block holds its SM slot (threads,
// registers and `working_set_bytes` of dynamic shared memory) while thread 0 sleeps
// `period_ns` per round; the other threads wait at the barrier.  No arithmetic, so
// no checksum: work = rounds.
__global__ void __launch_bounds__(1024) sleep_stress_kernel(DevStress *st, StressParams p) {
    __shared__ int s_k;
    __shared__ uint64_t s_t0;
    __shared__ int s_go[2];
    BlockCtl c;
    if (!block_enter(st, p, c, &s_k, &s_t0)) return;
    int64_t round = 0;
    for (;; ++round) {
        if (threadIdx.x == 0) {
            int go = round_decision(st, p, round, c);
            if (go) {
                const uint64_t until = ifr_gtimer() + p.period_ns;
                uint32_t it = 0;
                uint64_t now;
                while ((now = ifr_gtimer()) < until) {
                    if (now >= c.deadline) {
                        c.status = IFR_ERR_TIMEOUT;
                        go = 0;
                        break;
                    }
                    if (ifr_ld_volatile(&st->stop) || ++it > kMaxSpin) break;
                    sleep_toward(until - now);
                }
            }
            s_go[round & 1] = go;
        }
        __syncthreads();
        if (!s_go[round & 1]) break;
    }
    if (threadIdx.x == 0) write_log(p, st, c, round, (uint64_t)round, 0u, 0u);
}

// ------------------------------------------------------------------ shared memory
// Lane l = g*WAYS + r, iteration j: bank = g + (32/WAYS)*(j % WAYS),
// row = r + WAYS*(j / WAYS), word = 32*row + bank.  For a fixed j the WAYS lanes
// of a group hit one bank at WAYS distinct rows (WAYS-way conflict); over the 32
// iterations every lane visits its own 32 words once.  The conflict-free variant
// (WAYS = 1) uses 16-byte accesses instead (see the kernel); the checksum does not
// depend on which lane touches which word.
template <int WAYS>
__device__ __forceinline__ int smem_off(int j) {
    return 32 * WAYS * (j / WAYS) + (32 / WAYS) * (j % WAYS);
}

// 16-byte shared-memory load / store (conflict-free variant): a warp's request
// covers 512 contiguous bytes, four conflict-free wavefronts per instruction.
__device__ __forceinline__ void lds_v4(uint32_t addr, uint32_t (&v)[4]) {
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(addr)
                 : "memory");
}
__device__ __forceinline__ void sts_v4(uint32_t addr, const uint32_t (&v)[4]) {
    asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
                 : "memory");
}

template <int WAYS>
__global__ void __launch_bounds__(1024) smem_stress_kernel(DevStress *st, StressParams p) {
    extern __shared__ uint32_t s_arr[];
    __shared__ int s_k;
    __shared__ uint64_t s_t0;
    __shared__ int s_go[2];
    __shared__ uint32_t s_red[32];
    BlockCtl c;
    if (!block_enter(st, p, c, &s_k, &s_t0)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    volatile uint32_t *arr = s_arr + warp * 1024;
    const uint64_t s0 = p.seed << 32;
    for (int q = lane; q < 1024; q += 32)
        arr[q] = (uint32_t)ifr_splitmix64(s0, ((uint64_t)c.k * warps + warp) * 1024ull + q);
    __syncwarp();
    volatile uint32_t *mine = arr + 32 * (lane % WAYS) + lane / WAYS;
    int64_t round = 0, gpass = 0;
    for (;; ++round) {
        if (threadIdx.x == 0) s_go[round & 1] = round_decision(st, p, round, c);
        __syncthreads();
        if (!s_go[round & 1]) break;
#pragma unroll 1
        for (int pass = 0; pass < (WAYS >= kSmemPassesCF ? 1 : kSmemPassesCF / WAYS); ++pass, ++gpass) {
            // even passes update every word (LCG step), odd passes copy it back unchanged
            const uint32_t mul = (gpass & 1) ? 1u : 1664525u, add = (gpass & 1) ? 0u : 1013904223u;
            if constexpr (WAYS == 1) {
                // conflict-free: lane l owns words 4l..4l+3 of every 128-word row, moved
                // 16 bytes at a time, so the LSU issues one instruction per four
                // wavefronts instead of one per wavefront; every word is still read and
                // written once per pass
                const uint32_t base = (uint32_t)__cvta_generic_to_shared((const void *)arr) + 16u * lane;
#pragma unroll
                for (int h = 0; h < 8; h += 4) {
                    uint32_t v[4][4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) lds_v4(base + 512u * (h + i), v[i]);
                    if (!(gpass & 1)) {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int e = 0; e < 4; ++e) v[i][e] = v[i][e] * mul + add;
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) sts_v4(base + 512u * (h + i), v[i]);
                }
            } else if (gpass & 1) {
#pragma unroll
                for (int jb = 0; jb < 32; jb += 8) {
                    uint32_t v[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = mine[smem_off<WAYS>(jb + i)];
#pragma unroll
                    for (int i = 0; i < 8; ++i) mine[smem_off<WAYS>(jb + i)] = v[i];
                }
            } else {
#pragma unroll
                for (int jb = 0; jb < 32; jb += 8) {
                    uint32_t v[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = mine[smem_off<WAYS>(jb + i)];
#pragma unroll
                    for (int i = 0; i < 8; ++i) mine[smem_off<WAYS>(jb + i)] = v[i] * mul + add;
                }
            }
        }
    }
    __syncwarp();
    uint32_t acc = 0u;
    for (int q = lane; q < 1024; q += 32) acc ^= arr[q];
    uint32_t cs = ifr_block_xor(acc, s_red);
    if (threadIdx.x == 0)
        write_log(p, st, c, round, (uint64_t)round * (WAYS >= kSmemPassesCF ? 1 : kSmemPassesCF / WAYS) * 32, cs, 0u);
}

// ------------------------------------------------------------------ BF16 tensor pipe
// One 128-thread block per allowed SM holds A (128x64) and B (128x64, K-major)
// bf16 tiles of small integers in shared memory (128-byte swizzle) and a
// 128x128 fp32 accumulator in TMEM.  Thread 0 issues, per round, kTensorGroup
// tile products (4 tcgen05.mma of K = 16 each) into the zeroed accumulator, then
// commits and waits (bounded) on an mbarrier.  The accumulator ends as
// kTensorGroup * A B^T, exact in fp32; its XOR is the block checksum.
constexpr int kTensorGroup = 64;

__global__ void __launch_bounds__(128, 1) tensor_stress_kernel(DevStress *st, StressParams p) {
    extern __shared__ uint8_t t_smem_raw[];
    __shared__ int s_k;
    __shared__ uint64_t s_t0;
    __shared__ int s_go[2];
    __shared__ uint32_t s_red[32];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    BlockCtl c;
    if (!block_enter(st, p, c, &s_k, &s_t0)) return;
    uint8_t *base = (uint8_t *)(((uintptr_t)t_smem_raw + 1023u) & ~(uintptr_t)1023u);
    uint8_t *sA = base, *sB = base + 16384;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, 128);
        tc::tmem_relinquish();
    }
    const uint64_t s0 = p.seed << 32;
    for (int e = threadIdx.x; e < 8192; e += blockDim.x) {
        const uint32_t row = (uint32_t)e >> 6, col = (uint32_t)e & 63u;
        const uint64_t ua = ifr_splitmix64(s0, (uint64_t)c.k * 16384ull + (uint64_t)e);
        const uint64_t ub = ifr_splitmix64(s0, (uint64_t)c.k * 16384ull + 8192ull + (uint64_t)e);
        *(__nv_bfloat16 *)(sA + tc::sw128_offset(row, col)) = __int2bfloat16_rn((int)((ua >> 32) % 5u) - 2);
        *(__nv_bfloat16 *)(sB + tc::sw128_offset(row, col)) = __int2bfloat16_rn((int)((ub >> 32) % 5u) - 2);
    }
    tc::fence_proxy_async_smem();
    if (threadIdx.x == 0) {
        tc::mbar_init(&s_bar, 1);
        tc::fence_mbar_init();
        s_fail = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    const uint64_t adesc = tc::desc_sw128(tc::smem_u32(sA));
    const uint64_t bdesc = tc::desc_sw128(tc::smem_u32(sB));
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 128);
    int64_t round = 0;
    for (;; ++round) {
        if (threadIdx.x == 0) {
            int go = round_decision(st, p, round, c);
            if (go) {
                for (int g = 0; g < kTensorGroup; ++g)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc::mma_bf16(tmem, adesc + 2ull * kk, bdesc + 2ull * kk, idesc, (uint32_t)((g | kk) != 0));
                tc::mma_commit(&s_bar);
                if (!tc::mbar_wait(&s_bar, (uint32_t)(round & 1), c.deadline + 100000000ull)) {
                    c.status = IFR_ERR_TIMEOUT;
                    s_fail = 1;
                    go = 0;
                }
            }
            s_go[round & 1] = go;
        }
        __syncthreads();
        if (!s_go[round & 1]) break;
    }
    tc::fence_after();
    uint32_t acc = 0u;
    if (round > 0 && !s_fail) {
#pragma unroll 1
        for (int cc = 0; cc < 128; cc += 32) {
            uint32_t r[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, r);
            tc::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) acc ^= r[j];
        }
    }
    const uint32_t cs = ifr_block_xor(acc, s_red);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 128);
    }
    if (threadIdx.x == 0) write_log(p, st, c, round, (uint64_t)round * kTensorGroup, cs, 0u);
}

// ------------------------------------------------------------------ block scheduler
// Many short blocks of one warp.  Every block folds LCG^16(q ^ seed) into one of
// 64 XOR slots (q = launch * blocks + blockIdx); blocks on allowed SMs that see no
// stop request also stay resident for `sched_cycles` cycles.
__global__ void __launch_bounds__(32) sched_stress_kernel(DevStress *st, StressParams p, int launch_idx) {
    const uint64_t q = (uint64_t)launch_idx * (uint64_t)p.sched_blocks + blockIdx.x;
    int work = 0;
    if (threadIdx.x == 0) {
        const uint64_t now = ifr_gtimer();
        if (q == 0) {
            atomicExch((unsigned long long *)&st->t_origin, (unsigned long long)now);
            atomicAdd(&st->arrived, 1u);
        }
        uint32_t y = (uint32_t)q ^ (uint32_t)p.seed;
#pragma unroll
        for (int s = 0; s < kSchedLcgSteps; ++s) y = y * 1664525u + 1013904223u;
        atomicXor(&st->sched_xor[q & 63], y);
        uint64_t origin = *(volatile uint64_t *)&st->t_origin;
        if (origin == 0ull) origin = now;
        if (now > origin + p.deadline_ns) {
            atomicCAS(&st->status, 0, IFR_ERR_TIMEOUT);
        } else if (ifr_ld_volatile(&st->stop)) {
            // The chain was still being dispatched when the stop request came (the
            // sweeps request it after the victim's end): one block in 4096 records
            // when it saw it.  The sampled working-block ends alone can fall short of
            // the victim's end by the gap between two samples.  (A reduction whose
            // result is unused, so no block waits for a round trip; the samples are
            // sparse because every record of the chain goes to one address.)
            if ((q & 4095) == 0) atomicMin((unsigned long long *)&st->t_stop_seen, (unsigned long long)now);
        } else if (sm_allowed(p, ifr_smid())) {
            work = 1;
            if ((q & 255) == 0) atomicMin((unsigned long long *)&st->t_first_start, (unsigned long long)now);
        }
    }
    work = __shfl_sync(0xffffffffu, work, 0);
    if (!work) return;
    const long long t = clock64();
    uint32_t it = 0;
    while (clock64() - t < (long long)p.sched_cycles && ++it < kMaxSpin) {
    }
    if (threadIdx.x == 0) {
        atomicAdd(&st->sched_cnt[q & 63], 1u);
        if ((q & 255) == 0) atomicMax((unsigned long long *)&st->t_last_end, (unsigned long long)ifr_gtimer());
    }
}

// Residency wait on the victim stream.  A persistent stressor is resident once all
// its planned SM slots are claimed (`planned` > 0): the occupancy-sized grid's surplus
// blocks exit as soon as they arrive after that, and waiting for every one of them to
// arrive was seen on B300 to hold the victim back until the stressor had finished.
// A scheduler chain with allowed SMs (`first_work`) is resident once a recorded
// working block has started, so the victim never starts before the start the chain
// reports.  Otherwise (the zero-SM level) it waits for `expected` arrivals.
__device__ __forceinline__ bool stressor_ready(DevStress *st, uint32_t expected, uint32_t planned, int first_work) {
    if (first_work) return *(volatile unsigned long long *)&st->t_first_start != ~0ull;
    return planned > 0 ? ifr_ld_volatile(&st->active) >= planned : ifr_ld_volatile(&st->arrived) >= expected;
}

__global__ void wait_resident_kernel(DevStress *st, uint32_t expected, uint32_t planned, int first_work,
                                     uint64_t timeout_ns, DevTiming *tm) {
    if (threadIdx.x != 0) return;
    const uint64_t t0 = ifr_gtimer();
    uint32_t it = 0;
    while (!stressor_ready(st, expected, planned, first_work)) {
        if (ifr_gtimer() - t0 > timeout_ns || ++it > kMaxSpin) {
            if (tm) tm->status = IFR_ERR_NOT_RESIDENT;
            break;
        }
        __nanosleep(256);
    }
}

int kind_default_block(int kind) {
    switch (kind) {
        case IFR_S_SCHED: return 32;
        case IFR_S_FMA: return 128;
        case IFR_S_FP64: return 128;
        case IFR_S_SLEEP: return 128;
        case IFR_S_TENSOR: return 128;
        case IFR_S_SMEM_CF:
        case IFR_S_SMEM_32W: return 256;
        case IFR_S_L2:
        case IFR_S_HBM: return 512;
        default: return 128;
    }
}

int kind_default_bps(int kind) {
    switch (kind) {
        case IFR_S_FMA: return 2;
        case IFR_S_TENSOR: return 1;
        case IFR_S_SMEM_CF:
        case IFR_S_SMEM_32W: return 2;
        case IFR_S_L2:
        case IFR_S_HBM: return 2;
        default: return 1;
    }
}

template <int W>
const void *smem_fn() {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(smem_stress_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024 + 1024);
        attr = true;
    }
    return (const void *)smem_stress_kernel<W>;
}

// The sleep kernel may hold up to the device's opt-in shared memory per block.
const void *sleep_fn() {
    static bool attr = false;
    if (!attr) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        int static_bytes = 0;
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, sleep_stress_kernel) == cudaSuccess) static_bytes = (int)fa.sharedSizeBytes;
        attr = cudaFuncSetAttribute(sleep_stress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin - static_bytes) == cudaSuccess;
    }
    return (const void *)sleep_stress_kernel;
}

const void *smem_kernel_for(int ways) {
    switch (ways) {
        case 1: return smem_fn<1>();
        case 2: return smem_fn<2>();
        case 4: return smem_fn<4>();
        case 8: return smem_fn<8>();
        case 16: return smem_fn<16>();
        default: return smem_fn<32>();
    }
}

// Ring stages of the TMA-staged stream kernel: about 96 KiB of chunks per block
// (2 to kTmaMaxStages stages of block x 64 bytes), so two blocks of 512 threads fit
// on an SM with three stages each.
int tma_ring_stages(int block) {
    int n = (96 * 1024) / (block * 64);
    return n < 2 ? 2 : (n > kTmaMaxStages ? kTmaMaxStages : n);
}

const void *stream_tma_fn() {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(stream_stress_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * 1024 * 64);
        attr = true;
    }
    return (const void *)stream_stress_tma_kernel;
}

// Kernel, block, dynamic shared memory and grid of a persistent stressor launch.
struct StressShape {
    const void *fn;
    int block, smem, ways, bps, grid, occ;
};

StressShape stressor_shape(int num_sms, const ifr_stressor_cfg *cfg) {
    StressShape s;
    memset(&s, 0, sizeof s);
    const int kind = cfg->kind;
    s.block = kind == IFR_S_TENSOR ? 128 : (cfg->block ? cfg->block : kind_default_block(kind));
    s.bps = cfg->blocks_per_sm ? cfg->blocks_per_sm : kind_default_bps(kind);
    const int ilp = cfg->ilp ? cfg->ilp : 4;
    switch (kind) {
        case IFR_S_L2:
        case IFR_S_HBM:
            if (cfg->staging == 1) {
                s.fn = stream_tma_fn();
                s.smem = tma_ring_stages(s.block) * s.block * 64;
            } else {
                s.fn = stream_fn(s.block);
            }
            break;
        case IFR_S_FMA:
            s.fn = ilp == 1 ? (const void *)fma_stress_kernel<1>
                 : ilp == 2 ? (const void *)fma_stress_kernel<2>
                 : ilp == 4 ? (const void *)fma_stress_kernel<4>
                            : (const void *)fma_stress_kernel<8>;
            break;
        case IFR_S_FP64:
            s.fn = ilp == 1 ? (const void *)fp64_stress_kernel<1>
                 : ilp == 2 ? (const void *)fp64_stress_kernel<2>
                 : ilp == 4 ? (const void *)fp64_stress_kernel<4>
                            : (const void *)fp64_stress_kernel<8>;
            break;
        case IFR_S_SMEM_CF:
        case IFR_S_SMEM_32W:
            s.ways = cfg->smem_ways ? cfg->smem_ways : (kind == IFR_S_SMEM_CF ? 1 : 32);
            s.fn = smem_kernel_for(s.ways);
            s.smem = (s.block / 32) * 4096;
            break;
        case IFR_S_TENSOR:
            s.fn = (const void *)tensor_stress_kernel;
            s.smem = 32768 + 1024;
            break;
        case IFR_S_SLEEP:
            s.fn = sleep_fn();
            s.smem = (int)cfg->working_set_bytes;
            break;
        case IFR_S_SCHED:
            s.fn = (const void *)sched_stress_kernel;
            s.block = 32;
            s.grid = cfg->sched_blocks ? cfg->sched_blocks : 100000;
            return s;
        default: break;
    }
    // Launch enough blocks to fill every SM in the first wave (num_sms x occupancy):
    // each allowed SM then receives at least blocks_per_sm blocks to claim its
    // slots; the surplus blocks exit once the slots are taken.
    if (s.fn) {
        ifr_carveout(s.fn);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s.occ, s.fn, s.block, (size_t)s.smem) != cudaSuccess)
            s.occ = 0;
        if (s.occ > IFR_MAX_BPS) s.occ = IFR_MAX_BPS;
        s.grid = num_sms * (s.occ > s.bps ? s.occ : s.bps);
    } else {
        s.grid = num_sms * s.bps;
    }
    return s;
}

}  // namespace

extern "C" int ifr_stressor_profile(ifr_ctx *ctx, const ifr_stressor_cfg *cfg, ifr_kernel_profile *out) {
    if (!ctx || !cfg || !out || cfg->kind < 0 || cfg->kind >= IFR_S_COUNT) return IFR_ERR_ARG;
    memset(out, 0, sizeof *out);
    const StressShape s = stressor_shape(ctx->info.num_sms, cfg);
    cudaFuncAttributes fa;
    IFR_CUDA(cudaFuncGetAttributes(&fa, s.fn));
    int occ = 0;
    IFR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, s.fn, s.block, (size_t)s.smem));
    out->grid = s.grid;
    out->block = s.block;
    out->regs_per_thread = fa.numRegs;
    out->static_smem = (int32_t)fa.sharedSizeBytes;
    out->dynamic_smem = s.smem;
    out->max_blocks_per_sm = occ;
    out->tmem_cols = cfg->kind == IFR_S_TENSOR ? 128 : 0;
    out->uses_tensor = cfg->kind == IFR_S_TENSOR;
    out->sm_count = cfg->sm_count;
    out->blocks_per_sm = cfg->kind == IFR_S_SCHED ? 0 : s.bps;
    out->launches = cfg->kind == IFR_S_SCHED ? (cfg->sched_launches ? cfg->sched_launches : 64) : 1;
    return IFR_OK;
}

int ifr_stressor_expected_arrivals(const Slot &s) {
    return s.cfg.kind == IFR_S_SCHED ? 1 : s.grid;
}

static int validate_cfg(ifr_ctx *ctx, const ifr_stressor_cfg *c) {
    if (!c || c->kind < 0 || c->kind >= IFR_S_COUNT) return IFR_ERR_ARG;
    if (c->sm_count < 0 || c->sm_count > ctx->info.num_sms) return IFR_ERR_ARG;
    if (c->blocks_per_sm < 0 || c->blocks_per_sm > IFR_MAX_BPS) return IFR_ERR_ARG;
    if (c->block < 0 || c->block > 1024 || (c->block % 32) != 0) return IFR_ERR_ARG;
    if (c->duty < 0.f || c->duty > 1.f) return IFR_ERR_ARG;
    if (c->max_rounds < 0) return IFR_ERR_ARG;
    if ((c->kind == IFR_S_FMA || c->kind == IFR_S_FP64) &&
        !(c->ilp == 0 || c->ilp == 1 || c->ilp == 2 || c->ilp == 4 || c->ilp == 8))
        return IFR_ERR_ARG;
    if (c->kind == IFR_S_SMEM_CF || c->kind == IFR_S_SMEM_32W) {
        int w = c->smem_ways;
        if (!(w == 0 || w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32)) return IFR_ERR_ARG;
        int blk = c->block ? c->block : kind_default_block(c->kind);
        if (blk > 512) return IFR_ERR_ARG;  // 4 KiB per warp, at most 64 KiB per block
    }
    if (c->staging != 0 && (c->staging != 1 || (c->kind != IFR_S_L2 && c->kind != IFR_S_HBM))) return IFR_ERR_ARG;
    if (c->kind == IFR_S_L2 || c->kind == IFR_S_HBM) {
        int blk = c->block ? c->block : kind_default_block(c->kind);
        int64_t chunk = (int64_t)blk * 64;
        if (!c->buf || ((uintptr_t)c->buf & 15u)) return IFR_ERR_ARG;
        if (c->working_set_bytes < chunk || c->working_set_bytes % chunk) return IFR_ERR_ARG;
        if (c->working_set_bytes / chunk > (1ll << 30)) return IFR_ERR_ARG;  // 32-bit chunk positions
    }
    // one 128-thread block holds 128 TMEM columns; at most 2 per SM leave 256 of the
    // 512 columns for a GEMM victim block (so a TMEM allocation never waits long)
    if (c->kind == IFR_S_TENSOR && ((c->block != 0 && c->block != 128) || c->blocks_per_sm > 2)) return IFR_ERR_ARG;
    if (c->kind == IFR_S_SCHED && (c->sched_blocks < 0 || c->sched_launches < 0 || c->sched_cycles < 0))
        return IFR_ERR_ARG;
    if (c->kind == IFR_S_SLEEP &&
        (c->working_set_bytes < 0 || c->working_set_bytes > ctx->info.smem_per_block_optin - 1024 || c->period_ns < 0))
        return IFR_ERR_ARG;
    if (c->mask_mode == 1) {
        // the green context owning the launch stream confines the blocks
        if (!ctx->part_active) return IFR_ERR_UNSUPPORTED;
        const int most = ctx->part_sms_v > ctx->part_sms_s ? ctx->part_sms_v : ctx->part_sms_s;
        if (c->sm_count > most) return IFR_ERR_ARG;
    } else if (c->mask_mode == 2) {
        // explicit SM set: only ids of this device, exactly sm_count of them
        int bits = 0;
        for (int s = 0; s < IFR_MAX_SMS; ++s) {
            if (!((c->sm_mask[s >> 5] >> (s & 31)) & 1u)) continue;
            if (s >= ctx->info.num_sms) return IFR_ERR_ARG;
            ++bits;
        }
        if (bits != c->sm_count) return IFR_ERR_ARG;
    } else if (c->mask_mode != 0) {
        return IFR_ERR_ARG;
    }
    return IFR_OK;
}

int ifr_stressor_enqueue(ifr_ctx *ctx, const ifr_stressor_cfg *cfg, cudaStream_t stream, int slot, int record_events) {
    int rc = validate_cfg(ctx, cfg);
    if (rc != IFR_OK) return rc;
    rc = ifr_slot_prepare(ctx, slot);
    if (rc != IFR_OK) return rc;
    Slot &s = ctx->slots[slot];
    s.cfg = *cfg;
    const int num_sms = ctx->info.num_sms;
    const int kind = cfg->kind;
    StressParams p;
    memset(&p, 0, sizeof p);
    p.kind = kind;
    p.bps = cfg->blocks_per_sm ? cfg->blocks_per_sm : kind_default_bps(kind);
    if (cfg->mask_mode == 2)
        memcpy(p.mask, cfg->sm_mask, sizeof p.mask);
    else if (cfg->mask_mode == 1)
        ifr_compute_mask(num_sms, num_sms, p.mask);  // every SM id: the partition confines
    else
        ifr_compute_mask(num_sms, cfg->sm_count, p.mask);
    s.any_sm = 0;
    for (int i = 0; i < num_sms && i < IFR_MAX_SMS; ++i) s.any_sm |= (int)((p.mask[i >> 5] >> (i & 31)) & 1u);
    p.planned = cfg->sm_count * p.bps;
    p.seed = cfg->seed;
    p.max_rounds = cfg->max_rounds;
    p.deadline_ns = cfg->deadline_ns ? cfg->deadline_ns : 2000000000ull;
    p.duty = cfg->duty;
    p.period_ns = cfg->period_ns > 0 ? (uint32_t)cfg->period_ns : 100000u;
    p.duty_on_ns = (cfg->duty > 0.f && cfg->duty < 1.f) ? (uint32_t)((double)p.period_ns * (double)cfg->duty) : 0u;
    if (cfg->duty > 0.f && cfg->duty < 1.f && p.duty_on_ns == 0u) p.duty_on_ns = 1u;
    p.duty_inv_period = 1.0f / (float)p.period_ns;
    p.ilp = cfg->ilp ? cfg->ilp : 4;
    {
        // FMA constants: a = 1 - 2^-12 - (u0 >> 53) 2^-23, b = ((u1 >> 40) - 2^23) 2^-29
        // from outputs 0 and 1 of SplitMix64(seed << 32) (exact in fp32, |a| < 1)
        const uint64_t u0 = host_splitmix64(p.seed << 32, 0), u1 = host_splitmix64(p.seed << 32, 1);
        p.fma_a = (float)(1.0 - 0x1p-12 - (double)(u0 >> 53) * 0x1p-23);
        p.fma_b = (float)((double)((int64_t)(u1 >> 40) - (1 << 23)) * 0x1p-29);
        // FP64 multiplier: a = 1 - (1 + (u0 >> 54)) 2^-40 (exact in fp64, 0 < a < 1)
        p.fp64_a = 1.0 - (double)(1u + (unsigned)(u0 >> 54)) * 0x1p-40;
    }
    p.logs = s.d_logs;
    if (s.watch) {
        p.progress = ctx->d_progress;
        p.hol_ns = IFR_HOL_NS;
    }
    const int block = cfg->block ? cfg->block : kind_default_block(kind);
    s.block = block;
    s.planned = p.planned;
    s.launches = 1;
    const StressShape shape = stressor_shape(num_sms, cfg);
    const size_t sh = (size_t)shape.smem;
    const int ways = shape.ways;
    s.grid = shape.grid;
    ifr_carveout((const void *)stress_reset_kernel);
    stress_reset_kernel<<<1, 256, 0, stream>>>(s.d_state);
    IFR_CUDA(cudaGetLastError());
    IFR_CUDA(cudaEventRecord(s.ev_reset, stream));
    ctx->kernel_launches += (kind == IFR_S_SCHED) ? 1 : 2;
    if (record_events) IFR_CUDA(cudaEventRecord(s.ev_start, stream));
    const dim3 grid(s.grid), blk(block);
    switch (kind) {
        case IFR_S_L2:
        case IFR_S_HBM:
            p.buf = (const int4 *)cfg->buf;
            p.n_chunks = cfg->working_set_bytes / ((int64_t)block * 64);
            p.ring = tma_ring_stages(block);
            if (cfg->staging == 1)
                stream_stress_tma_kernel<<<grid, blk, sh, stream>>>(s.d_state, p);
            else
                launch_stream(s.grid, block, stream, s.d_state, p);
            break;
        case IFR_S_FMA:
            switch (p.ilp) {
                case 1: fma_stress_kernel<1><<<grid, blk, 0, stream>>>(s.d_state, p); break;
                case 2: fma_stress_kernel<2><<<grid, blk, 0, stream>>>(s.d_state, p); break;
                case 4: fma_stress_kernel<4><<<grid, blk, 0, stream>>>(s.d_state, p); break;
                default: fma_stress_kernel<8><<<grid, blk, 0, stream>>>(s.d_state, p); break;
            }
            break;
        case IFR_S_FP64:
            switch (p.ilp) {
                case 1: fp64_stress_kernel<1><<<grid, blk, 0, stream>>>(s.d_state, p); break;
                case 2: fp64_stress_kernel<2><<<grid, blk, 0, stream>>>(s.d_state, p); break;
                case 4: fp64_stress_kernel<4><<<grid, blk, 0, stream>>>(s.d_state, p); break;
                default: fp64_stress_kernel<8><<<grid, blk, 0, stream>>>(s.d_state, p); break;
            }
            break;
        case IFR_S_SMEM_CF:
        case IFR_S_SMEM_32W:
            p.ways = ways;
            switch (ways) {
                case 1: smem_stress_kernel<1><<<grid, blk, sh, stream>>>(s.d_state, p); break;
                case 2: smem_stress_kernel<2><<<grid, blk, sh, stream>>>(s.d_state, p); break;
                case 4: smem_stress_kernel<4><<<grid, blk, sh, stream>>>(s.d_state, p); break;
                case 8: smem_stress_kernel<8><<<grid, blk, sh, stream>>>(s.d_state, p); break;
                case 16: smem_stress_kernel<16><<<grid, blk, sh, stream>>>(s.d_state, p); break;
                default: smem_stress_kernel<32><<<grid, blk, sh, stream>>>(s.d_state, p); break;
            }
            break;
        case IFR_S_TENSOR:
            s.block = 128;
            tensor_stress_kernel<<<grid, 128, sh, stream>>>(s.d_state, p);
            break;
        case IFR_S_SLEEP:
            sleep_stress_kernel<<<grid, blk, sh, stream>>>(s.d_state, p);
            break;
        case IFR_S_SCHED: {
            p.sched_blocks = cfg->sched_blocks ? cfg->sched_blocks : 100000;
            p.sched_cycles = cfg->sched_cycles ? cfg->sched_cycles : 100;
            s.launches = cfg->sched_launches ? cfg->sched_launches : 64;
            s.grid = p.sched_blocks;
            s.block = 32;
            s.planned = p.sched_blocks;
            ifr_carveout((const void *)sched_stress_kernel);
            for (int l = 0; l < s.launches; ++l) sched_stress_kernel<<<p.sched_blocks, 32, 0, stream>>>(s.d_state, p, l);
            ctx->kernel_launches += (uint64_t)s.launches;
            break;
        }
        default: return IFR_ERR_ARG;
    }
    IFR_CUDA(cudaGetLastError());
    if (record_events) IFR_CUDA(cudaEventRecord(s.ev_end, stream));
    s.stream = stream;
    s.in_use = 1;
    s.finished = 0;
    return IFR_OK;
}

int ifr_enqueue_wait_resident(ifr_ctx *ctx, int slot, cudaStream_t stream, DevTiming *tm, uint64_t timeout_ns) {
    Slot &s = ctx->slots[slot];
    // the wait must not start before the stressor's state reset (cross-stream edge)
    IFR_CUDA(cudaStreamWaitEvent(stream, s.ev_reset, 0));
    ifr_carveout((const void *)wait_resident_kernel);
    const uint32_t planned = s.cfg.kind == IFR_S_SCHED ? 0u : (uint32_t)s.planned;
    const int first_work = s.cfg.kind == IFR_S_SCHED && s.any_sm;
    wait_resident_kernel<<<1, 32, 0, stream>>>(s.d_state, (uint32_t)ifr_stressor_expected_arrivals(s), planned,
                                               first_work, timeout_ns, tm);
    IFR_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    return IFR_OK;
}

int ifr_enqueue_stop(ifr_ctx *ctx, int slot, cudaStream_t stream) {
    Slot &s = ctx->slots[slot];
    IFR_CUDA(cudaMemcpyAsync(&s.d_state->stop, ctx->h_one, sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
    return IFR_OK;
}

int ifr_stressor_collect(ifr_ctx *ctx, int slot) {
    Slot &s = ctx->slots[slot];
    DevStress h;
    IFR_CUDA(cudaMemcpy(&h, s.d_state, sizeof h, cudaMemcpyDeviceToHost));
    ifr_stressor_result &r = s.result;
    memset(&r, 0, sizeof r);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s.ev_start, s.ev_end) != cudaSuccess) {
        ms = 0.f;
        cudaGetLastError();
    }
    r.elapsed_ms = ms;
    r.status = h.status;
    r.planned_active = s.planned;
    if (s.cfg.kind == IFR_S_SCHED) {
        uint32_t x = 0u;
        uint64_t cnt = 0;
        for (int i = 0; i < 64; ++i) {
            x ^= h.sched_xor[i];
            cnt += h.sched_cnt[i];
        }
        r.checksum = x;
        r.work = cnt;
        r.rounds = cnt;
        r.blocks_launched = s.grid * s.launches;
        r.blocks_active = cnt > 0x7fffffffull ? 0x7fffffff : (int32_t)cnt;
        r.sms_used = 0;
        if (cnt > 0) {
            r.t_start_ns = r.t_start_last_ns = h.t_first_start;
            const bool seen = h.t_stop_seen != ~0ull && h.t_stop_seen > h.t_last_end;
            r.t_end_ns = r.t_end_first_ns = seen ? h.t_stop_seen : h.t_last_end;
        }
        s.h_nlogs = 0;
        s.finished = 1;
        return IFR_OK;
    }
    int n = (int)(h.active < (uint32_t)s.planned ? h.active : (uint32_t)s.planned);
    if (n > s.log_cap) n = s.log_cap;
    if (n > 0) IFR_CUDA(cudaMemcpy(s.h_logs, s.d_logs, sizeof(ifr_block_log) * (size_t)n, cudaMemcpyDeviceToHost));
    s.h_nlogs = n;
    r.blocks_launched = s.grid;
    r.blocks_active = n;
    uint32_t used[IFR_MAX_SMS / 32] = {0};
    if (n > 0) {
        r.t_start_ns = ~0ull;
        r.t_end_first_ns = ~0ull;
    }
    for (int i = 0; i < n; ++i) {
        const ifr_block_log &L = s.h_logs[i];
        r.checksum ^= L.checksum;
        r.rounds += L.rounds;
        r.work += L.work;
        if (L.t_start_ns < r.t_start_ns) r.t_start_ns = L.t_start_ns;
        if (L.t_start_ns > r.t_start_last_ns) r.t_start_last_ns = L.t_start_ns;
        if (L.t_end_ns < r.t_end_first_ns) r.t_end_first_ns = L.t_end_ns;
        if (L.t_end_ns > r.t_end_ns) r.t_end_ns = L.t_end_ns;
        if (L.smid < IFR_MAX_SMS) used[L.smid >> 5] |= 1u << (L.smid & 31);
        if (L.status != 0 && r.status == 0) r.status = L.status;
    }
    for (int i = 0; i < IFR_MAX_SMS / 32; ++i) r.sms_used += __builtin_popcount(used[i]);
    s.finished = 1;
    return IFR_OK;
}

// ------------------------------------------------------------------ public API
extern "C" int ifr_stressor_launch(ifr_ctx *ctx, const ifr_stressor_cfg *cfg, void *stream, int *handle_out) {
    if (!ctx || !cfg || !handle_out) return IFR_ERR_ARG;
    int slot = ifr_slot_alloc(ctx);
    if (slot < 0) return slot;
    ctx->slots[slot].watch = 0;
    int rc = ifr_stressor_enqueue(ctx, cfg, stream ? (cudaStream_t)stream : ctx->s_stress, slot);
    if (rc != IFR_OK) return rc;
    *handle_out = slot;
    return IFR_OK;
}

static bool valid_handle(ifr_ctx *ctx, int h) { return ctx && h >= 0 && h < IFR_SLOTS && ctx->slots[h].in_use; }

extern "C" int ifr_stressor_stop(ifr_ctx *ctx, int handle, void *stream) {
    if (!valid_handle(ctx, handle)) return IFR_ERR_ARG;
    return ifr_enqueue_stop(ctx, handle, stream ? (cudaStream_t)stream : ctx->s_ctrl);
}

extern "C" int ifr_stressor_wait(ifr_ctx *ctx, int handle, int timeout_ms, ifr_stressor_result *out) {
    if (!valid_handle(ctx, handle)) return IFR_ERR_ARG;
    Slot &s = ctx->slots[handle];
    if (!s.finished) {
        const int limit = timeout_ms > 0 ? timeout_ms : 10000;
        cudaEvent_t ev = s.ev_end;
        int waited_us = 0;
        cudaError_t q;
        while ((q = cudaEventQuery(ev)) == cudaErrorNotReady) {
            if (waited_us >= limit * 1000) {
                ifr_enqueue_stop(ctx, handle, ctx->s_ctrl);
                cudaEventSynchronize(ev);  // the kernels' own deadlines bound this wait
                int rc = ifr_stressor_collect(ctx, handle);
                if (out) *out = s.result;
                return rc != IFR_OK ? rc : IFR_ERR_TIMEOUT;
            }
            struct timespec ts = {0, 50000};
            nanosleep(&ts, nullptr);
            waited_us += 50;
        }
        if (q != cudaSuccess) return ifr_cuda_fail(q, "cudaEventQuery(stressor end)", __FILE__, __LINE__);
        int rc = ifr_stressor_collect(ctx, handle);
        if (rc != IFR_OK) return rc;
    }
    if (out) *out = s.result;
    return IFR_OK;
}

extern "C" int ifr_stressor_block_logs(ifr_ctx *ctx, int handle, ifr_block_log *out, int cap, int *n_out) {
    if (!valid_handle(ctx, handle) || !n_out || (cap > 0 && !out)) return IFR_ERR_ARG;
    Slot &s = ctx->slots[handle];
    if (!s.finished) return IFR_ERR_ARG;
    *n_out = s.h_nlogs;
    if (cap < s.h_nlogs) return IFR_ERR_CAPACITY;
    memcpy(out, s.h_logs, sizeof(ifr_block_log) * (size_t)s.h_nlogs);
    return IFR_OK;
}

extern "C" int ifr_stressor_release(ifr_ctx *ctx, int handle) {
    if (!valid_handle(ctx, handle)) return IFR_ERR_ARG;
    Slot &s = ctx->slots[handle];
    if (!s.finished) {
        ifr_stressor_result r;
        int rc = ifr_stressor_wait(ctx, handle, 0, &r);
        if (rc != IFR_OK && rc != IFR_ERR_TIMEOUT) return rc;
    }
    s.in_use = 0;
    return IFR_OK;
}

// ------------------------------------------------------------------ allocation-free variant
// Control state (stop flag, counters, per-SM claims) of ifr_stream_stressor_noalloc.
// It lives in this file-scope device array, so the entry point needs no
// cudaMalloc; every GPU that loads the library keeps these bytes until exit.
// All calls share the array: calls whose kernels overlap on the GPU race on it.
#define IFR_NOALLOC_SCRATCH_BYTES 4096
static __device__ __align__(256) unsigned char g_noalloc_scratch[IFR_NOALLOC_SCRATCH_BYTES];
static_assert(sizeof(DevStress) <= IFR_NOALLOC_SCRATCH_BYTES, "scratch array too small for DevStress");

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoallocMaxDevices];  // device address of the array, per device (host cache)

__global__ void noalloc_logs_clear_kernel(ifr_block_log *logs, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        ifr_block_log L;
        memset(&L, 0, sizeof L);
        L.index = -1;
        logs[i] = L;
    }
}
}  // namespace

extern "C" int ifr_stream_stressor_noalloc(int kind, const void *buf, int64_t working_set_bytes, int sm_count,
                                           int blocks_per_sm, int block, int64_t max_rounds, uint64_t deadline_ns,
                                           void *stream, ifr_block_log *logs_out, int logs_cap) {
    if (kind != IFR_S_L2 && kind != IFR_S_HBM) return IFR_ERR_ARG;
    if (!buf || ((uintptr_t)buf & 15u) || !logs_out || ((uintptr_t)logs_out & 7u)) return IFR_ERR_ARG;
    if (block <= 0 || block > 1024 || block % 32) return IFR_ERR_ARG;
    const int64_t chunk = (int64_t)block * 64;
    if (working_set_bytes < chunk || working_set_bytes % chunk) return IFR_ERR_ARG;
    if (working_set_bytes / chunk > (1ll << 30)) return IFR_ERR_ARG;  // 32-bit chunk positions
    if (max_rounds <= 0 || blocks_per_sm <= 0 || blocks_per_sm > IFR_MAX_BPS) return IFR_ERR_ARG;
    int dev = 0, num_sms = 0;
    IFR_CUDA(cudaGetDevice(&dev));
    IFR_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    // the array holds per-SM claim counters for at most IFR_MAX_SMS SMs
    if (num_sms > IFR_MAX_SMS || dev >= kNoallocMaxDevices) return IFR_ERR_CAPACITY;
    if (sm_count <= 0 || sm_count > num_sms) return IFR_ERR_ARG;
    if ((int64_t)sm_count * blocks_per_sm > logs_cap) return IFR_ERR_CAPACITY;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            // first call on this device: look up the array's device address with
            // the device current (host code cannot use the symbol itself), and load
            // the three kernels now rather than lazily at their first launch
            void *ptr = nullptr;
            IFR_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
            const void *fns[] = {(const void *)stress_reset_kernel, stream_fn(128), stream_fn(256), stream_fn(512), stream_fn(0),
                                 (const void *)noalloc_logs_clear_kernel};
            for (const void *f : fns) {
                int rc = ifr_preload(f);
                if (rc) return rc;
            }
            g_noalloc_addr[dev] = ptr;
        }
        scratch = g_noalloc_addr[dev];
    }
    DevStress *st = (DevStress *)scratch;
    cudaStream_t s = (cudaStream_t)stream;
    StressParams p;
    memset(&p, 0, sizeof p);
    p.kind = kind;
    p.bps = blocks_per_sm;
    ifr_compute_mask(num_sms, sm_count, p.mask);
    p.planned = sm_count * blocks_per_sm;
    p.max_rounds = max_rounds;
    p.deadline_ns = deadline_ns ? deadline_ns : 2000000000ull;
    p.duty = 1.f;
    p.period_ns = 100000u;
    p.duty_on_ns = 0u;
    p.logs = logs_out;
    p.buf = (const int4 *)buf;
    p.n_chunks = working_set_bytes / chunk;
    ifr_carveout(stream_fn(block));
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, stream_fn(block), block, 0) != cudaSuccess)
        occ = 0;
    if (occ > IFR_MAX_BPS) occ = IFR_MAX_BPS;
    const int grid = num_sms * (occ > blocks_per_sm ? occ : blocks_per_sm);
    // the previous call's counters and claims are still in the array: clear them
    stress_reset_kernel<<<1, 256, 0, s>>>(st);
    noalloc_logs_clear_kernel<<<(p.planned + 127) / 128, 128, 0, s>>>(logs_out, p.planned);
    launch_stream(grid, block, s, st, p);
    IFR_CUDA(cudaGetLastError());
    return IFR_OK;
}

int ifr_preload_stressors() {
    const void *fns[] = {
        (const void *)stress_reset_kernel, stream_fn(128), stream_fn(256), stream_fn(512), stream_fn(0), stream_tma_fn(),
        (const void *)fma_stress_kernel<1>, (const void *)fma_stress_kernel<2>, (const void *)fma_stress_kernel<4>,
        (const void *)fma_stress_kernel<8>, (const void *)fp64_stress_kernel<1>, (const void *)fp64_stress_kernel<2>,
        (const void *)fp64_stress_kernel<4>, (const void *)fp64_stress_kernel<8>, smem_kernel_for(1),
        smem_kernel_for(2), smem_kernel_for(4), smem_kernel_for(8), smem_kernel_for(16), smem_kernel_for(32),
        (const void *)tensor_stress_kernel, (const void *)sched_stress_kernel, sleep_fn(),
        (const void *)wait_resident_kernel, (const void *)noalloc_logs_clear_kernel};
    for (const void *f : fns) {
        int rc = ifr_preload(f);
        if (rc) return rc;
    }
    return IFR_OK;
}
