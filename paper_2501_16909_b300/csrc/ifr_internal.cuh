// Internal declarations shared by the libifr translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ifr.h"

#define IFR_SLOTS 8
#define IFR_MAX_BPS 32

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint64_t ifr_gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ifr_smid() {
    uint32_t s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}
__device__ __forceinline__ uint32_t ifr_ld_volatile(const uint32_t *p) {
    return *(const volatile uint32_t *)p;
}
__device__ __forceinline__ uint32_t ifr_rotl(uint32_t x, uint32_t r) {
    return __funnelshift_l(x, x, r & 31u);
}
// SplitMix64 (Steele, Lea, Flood 2014): output i of the stream started at s0.
__device__ __forceinline__ uint64_t ifr_splitmix64(uint64_t s0, uint64_t i) {
    uint64_t z = s0 + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint32_t ifr_warp_xor(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Block-wide XOR; every thread must call it; result valid in thread 0.
__device__ __forceinline__ uint32_t ifr_block_xor(uint32_t v, uint32_t *scratch32) {
    v = ifr_warp_xor(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch32[warp] = v;
    __syncthreads();
    uint32_t r = 0;
    if (warp == 0) {
        r = (lane < (int)((blockDim.x + 31) >> 5)) ? scratch32[lane] : 0u;
        r = ifr_warp_xor(r);
    }
    return r;
}

// ---------------------------------------------------------------- device state
// One per stressor slot; reset by a kernel before each launch.
struct DevStress {
    uint32_t stop;        // 1 = stop requested
    uint32_t arrived;     // grid blocks that passed entry (after their SM claim)
    uint32_t active;      // blocks that claimed an SM slot (claim order = active index)
    int32_t status;       // first error
    uint64_t t_origin;    // SCHED: first block start (deadline origin)
    uint64_t t_first_start, t_last_end;  // SCHED sampled window
    uint64_t t_stop_seen;                // SCHED: earliest sampled block that saw the stop request (~0: none)
    uint32_t sm_claim[IFR_MAX_SMS];
    uint32_t sched_xor[64];
    uint32_t sched_cnt[64];
};

// One per victim measurement.
struct DevTiming {
    uint64_t t_min, t_max;
    uint32_t blocks;
    int32_t status;
    uint32_t sm_bits[IFR_MAX_SMS / 32];
    uint64_t *progress;  // context-wide "last victim block entry/exit" (%globaltimer)
    uint32_t tile_next;  // GEMM: next output tile to hand out (0 between launches)
    uint32_t tile_done;  // GEMM: CTAs of the running launch that have finished
    uint32_t done;       // grouped launches: rows (GEMM: tile-warps) of this victim finished
};

// Kernel parameters of a stressor launch (passed by value).
struct StressParams {
    int32_t kind;
    int32_t planned;      // planned active blocks (work-split stride)
    int32_t bps;          // blocks per allowed SM
    uint32_t mask[IFR_MAX_SMS / 32];
    uint64_t seed;
    int64_t max_rounds;
    uint64_t deadline_ns; // per-block, relative to its own start
    float duty;
    uint32_t period_ns;
    uint32_t duty_on_ns;  // active part of each period (0 = no duty cycle)
    float duty_inv_period; // 1 / period_ns
    const int4 *buf;      // L2/HBM
    int64_t n_chunks;     // L2/HBM chunks (chunk = blockDim * 4 int4)
    int32_t ring;         // L2/HBM with TMA staging: shared-memory ring stages
    int32_t ilp;          // FMA
    float fma_a, fma_b;   // FMA multiplier and addend (launch-wide)
    double fp64_a;        // FP64 multiplier (launch-wide)
    int32_t ways;         // SMEM
    int32_t sched_blocks, sched_cycles;
    ifr_block_log *logs;
    const uint64_t *progress;  // victim progress word to watch (NULL = no watch)
    uint64_t hol_ns;           // give up when no victim progress for this long
};

// ---------------------------------------------------------------- host context
struct Slot {
    int in_use;
    int finished;
    ifr_stressor_cfg cfg;
    DevStress *d_state;
    ifr_block_log *d_logs;
    int log_cap;
    cudaEvent_t ev_start, ev_end;
    cudaEvent_t ev_reset;  // recorded after the state reset; victims wait on it
    int grid, block, planned, launches;
    int watch;             // watch the context's victim-progress word (sweeps)
    int any_sm;            // the launch's SM mask allows at least one SM of the device
    cudaStream_t stream;
    ifr_stressor_result result;
    ifr_block_log *h_logs;
    int h_nlogs;
};

struct ifr_ctx {
    int device;
    ifr_device_info info;
    cudaStream_t s_stress, s_victim, s_ctrl;
    Slot slots[IFR_SLOTS];
    DevTiming *d_timing;
    int timing_cap;
    uint32_t *h_one;  // pinned, holds 1 (stop writes)
    cudaEvent_t ev_a, ev_b;
    uint64_t kernel_launches;  // kernels enqueued (graph replays add their kernel nodes)
    uint64_t *d_progress;      // victim progress word (device)
    // green-context split (ifr_partition): the victim / stressor streams above are
    // the partitions' streams while it is active; the originals are kept here
    int part_active;
    int part_sms_v, part_sms_s;
    void *green_v, *green_s;   // CUgreenCtx
    cudaStream_t own_victim, own_stress;
    // GEMM variant 3: partial tiles of a split last wave and their arrival counters
    float *gemm_ws;
    size_t gemm_ws_bytes;
    uint32_t *gemm_cnt;
    size_t gemm_cnt_n;
    int64_t gemm_cnt_key;  // split the counters were zeroed for (-1: zero before the next use)
};

// Prefer the maximum shared-memory carveout for every kernel of the library so
// that stressor and victim blocks can share an SM without a carveout switch
// (the paper sets the same split for the same reason, Sec. 4.4.2).
void ifr_carveout(const void *func);
// Load a kernel now (and set its carveout).  With lazy module loading a kernel's
// first launch can wait for the device to drain, which would hold a victim back
// behind a running stressor; ifr_init therefore loads every kernel of the library.
int ifr_preload(const void *func);
int ifr_preload_stressors();
int ifr_preload_victims();
int ifr_preload_gemm();
int ifr_preload_sweep();
int ifr_preload_mlp();
#define IFR_HOL_NS 50000000ull  // 50 ms without victim progress = head-of-line blocked

// ---------------------------------------------------------------- internal API
#define IFR_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ifr_cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

int ifr_cuda_fail(cudaError_t e, const char *what, const char *file, int line);
const char *ifr_last_cuda_error();

// stressors (ifr_stressors.cu)
int ifr_stressor_enqueue(ifr_ctx *ctx, const ifr_stressor_cfg *cfg, cudaStream_t stream, int slot,
                         int record_events = 1);
int ifr_stressor_collect(ifr_ctx *ctx, int slot);  // after completion: fills slot result + host logs
int ifr_stressor_expected_arrivals(const Slot &s);
int ifr_slot_alloc(ifr_ctx *ctx);
int ifr_slot_prepare(ifr_ctx *ctx, int slot);
void ifr_compute_mask(int num_sms, int sm_count, uint32_t *mask);
int ifr_enqueue_wait_resident(ifr_ctx *ctx, int slot, cudaStream_t stream, DevTiming *tm, uint64_t timeout_ns);
int ifr_enqueue_stop(ifr_ctx *ctx, int slot, cudaStream_t stream);


// victims (ifr_victims.cu)
int ifr_victim_validate(ifr_ctx *ctx, const ifr_victim_cfg *cfg);
int ifr_victim_enqueue(ifr_ctx *ctx, const ifr_victim_cfg *cfg, cudaStream_t stream, DevTiming *tm);
int ifr_timing_reset(DevTiming *tm, int n, cudaStream_t stream, uint64_t *progress);
void ifr_timing_to_host(const DevTiming &d, int repeats, ifr_timing *out);
int ifr_ensure_timing(ifr_ctx *ctx, int n);

// Launch shape and algorithmic work of one victim launch.
// Grouped victims (graph-batched sweeps with grouping): the grouping key of a victim
// (victims with equal keys > 0 may share one persistent launch; 0 = launched alone)
// and the grouped launch of n such victims, victim i stamping into tms[i].
#define IFR_GROUP_MAX 16
int ifr_victim_group_key(ifr_ctx *ctx, const ifr_victim_cfg *cfg);
int ifr_victims_enqueue_group(ifr_ctx *ctx, const ifr_victim_cfg *const *victims, DevTiming *const *tms, int n,
                              cudaStream_t stream);

struct VictimShape {
    const void *fn;
    int grid, block, smem, tmem_cols, uses_tensor;
    double bytes, flops;
};
int ifr_victim_shape(ifr_ctx *ctx, const ifr_victim_cfg *cfg, VictimShape *s);

// GEMM (ifr_gemm.cu)
int ifr_gemm_enqueue(ifr_ctx *ctx, const ifr_victim_cfg *cfg, cudaStream_t stream, DevTiming *tm);
int ifr_gemm_shape(const ifr_victim_cfg *cfg, VictimShape *s);
int ifr_gemm_group_key(const ifr_victim_cfg *cfg);
int ifr_gemm_enqueue_group(ifr_ctx *ctx, const ifr_victim_cfg *const *victims, DevTiming *const *tms, int n,
                           cudaStream_t stream);
void ifr_gemm_forget_split(ifr_ctx *ctx);
