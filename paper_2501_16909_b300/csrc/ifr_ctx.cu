// Context: device query, streams, stressor slots, error reporting.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <unordered_set>

#include "ifr_internal.cuh"

static thread_local char g_last_err[512];

int ifr_cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_last_err, sizeof g_last_err, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return IFR_ERR_CUDA;
}

const char *ifr_last_cuda_error() { return g_last_err; }

extern "C" const char *ifr_strerror(int status) {
    switch (status) {
        case IFR_OK: return "ok";
        case IFR_ERR_ARG: return "invalid argument";
        case IFR_ERR_CUDA: return g_last_err[0] ? g_last_err : "CUDA call failed";
        case IFR_ERR_TIMEOUT: return "wait reached its deadline";
        case IFR_ERR_NOT_RESIDENT: return "stressor not resident before the victim started";
        case IFR_ERR_LAUNCH: return "kernel launch rejected";
        case IFR_ERR_BOUNDS: return "index out of range (checked build)";
        case IFR_ERR_UNSUPPORTED: return "unsupported on this device";
        case IFR_ERR_NOMEM: return "scratch allocation failed";
        case IFR_ERR_CAPACITY: return "capacity exceeded";
        case IFR_ERR_INVALID_CELL: return "measurement violated the constant-interference rule";
        case IFR_ERR_HOL: return "victim could not become co-resident with the stressor (head-of-line blocking)";
        default: return "unknown status";
    }
}

extern "C" int ifr_abi_version(void) { return IFR_ABI_VERSION; }

extern "C" int ifr_init(int device, ifr_ctx **out) {
    if (!out) return IFR_ERR_ARG;
    *out = nullptr;
    int n = 0;
    IFR_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return IFR_ERR_ARG;
    IFR_CUDA(cudaSetDevice(device));
    cudaDeviceProp p;
    IFR_CUDA(cudaGetDeviceProperties(&p, device));
    if (p.major != 10) return IFR_ERR_UNSUPPORTED;
    ifr_ctx *c = (ifr_ctx *)calloc(1, sizeof(ifr_ctx));
    if (!c) return IFR_ERR_NOMEM;
    c->device = device;
    c->gemm_cnt_key = -1;
    ifr_device_info &d = c->info;
    d.device = device;
    d.num_sms = p.multiProcessorCount;
    d.cc_major = p.major;
    d.cc_minor = p.minor;
    d.l2_bytes = p.l2CacheSize;
    d.smem_per_sm = (int32_t)p.sharedMemPerMultiprocessor;
    d.smem_per_block_optin = (int32_t)p.sharedMemPerBlockOptin;
    d.regs_per_sm = p.regsPerMultiprocessor;
    d.max_threads_per_sm = p.maxThreadsPerMultiProcessor;
    d.max_blocks_per_sm = p.maxBlocksPerMultiProcessor;
    int clk = 0, mclk = 0, bus = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device);
    cudaDeviceGetAttribute(&mclk, cudaDevAttrMemoryClockRate, device);
    cudaDeviceGetAttribute(&bus, cudaDevAttrGlobalMemoryBusWidth, device);
    d.sm_clock_khz = clk;
    d.mem_clock_khz = mclk;
    d.mem_bus_width_bits = bus;
    d.global_mem_bytes = (int64_t)p.totalGlobalMem;
    strncpy(d.name, p.name, sizeof d.name - 1);
    if (d.num_sms > IFR_MAX_SMS) {
        free(c);
        return IFR_ERR_UNSUPPORTED;
    }
    int rc = IFR_OK;
#define TRY(x)                                              \
    do {                                                    \
        cudaError_t e_ = (x);                               \
        if (e_ != cudaSuccess) {                            \
            rc = ifr_cuda_fail(e_, #x, __FILE__, __LINE__); \
            goto fail;                                      \
        }                                                   \
    } while (0)
    TRY(cudaStreamCreateWithFlags(&c->s_stress, cudaStreamNonBlocking));
    TRY(cudaStreamCreateWithFlags(&c->s_victim, cudaStreamNonBlocking));
    TRY(cudaStreamCreateWithFlags(&c->s_ctrl, cudaStreamNonBlocking));
    TRY(cudaHostAlloc((void **)&c->h_one, sizeof(uint32_t), cudaHostAllocDefault));
    *c->h_one = 1u;
    TRY(cudaEventCreate(&c->ev_a));
    TRY(cudaEventCreate(&c->ev_b));
    TRY(cudaMalloc(&c->d_progress, sizeof(uint64_t)));
    TRY(cudaMemset(c->d_progress, 0, sizeof(uint64_t)));
    rc = ifr_ensure_timing(c, 64);
    if (rc != IFR_OK) goto fail;
    if ((rc = ifr_preload_stressors()) || (rc = ifr_preload_victims()) || (rc = ifr_preload_gemm()) ||
        (rc = ifr_preload_sweep()) || (rc = ifr_preload_mlp()))
        goto fail;
#undef TRY
    *out = c;
    return IFR_OK;
fail:
    ifr_shutdown(c);
    return rc;
}

int ifr_ensure_timing(ifr_ctx *ctx, int n) {
    if (n <= ctx->timing_cap) return IFR_OK;
    if (ctx->d_timing) {
        cudaDeviceSynchronize();
        cudaFree(ctx->d_timing);
        ctx->d_timing = nullptr;
        ctx->timing_cap = 0;
    }
    IFR_CUDA(cudaMalloc(&ctx->d_timing, sizeof(DevTiming) * (size_t)n));
    IFR_CUDA(cudaMemset(ctx->d_timing, 0, sizeof(DevTiming) * (size_t)n));
    ctx->timing_cap = n;
    return IFR_OK;
}

static void slot_free(Slot &s) {
    if (s.d_state) cudaFree(s.d_state);
    if (s.d_logs) cudaFree(s.d_logs);
    if (s.ev_start) cudaEventDestroy(s.ev_start);
    if (s.ev_end) cudaEventDestroy(s.ev_end);
    if (s.ev_reset) cudaEventDestroy(s.ev_reset);
    free(s.h_logs);
    memset(&s, 0, sizeof s);
}

extern "C" void ifr_shutdown(ifr_ctx *ctx) {
    if (!ctx) return;
    // stop anything still running, then wait (bounded by the kernels' own deadlines)
    for (int i = 0; i < IFR_SLOTS; ++i)
        if (ctx->slots[i].in_use && ctx->slots[i].d_state && ctx->h_one)
            cudaMemcpyAsync(&ctx->slots[i].d_state->stop, ctx->h_one, 4, cudaMemcpyHostToDevice, ctx->s_ctrl);
    cudaDeviceSynchronize();
    ifr_partition_release(ctx);
    for (int i = 0; i < IFR_SLOTS; ++i) slot_free(ctx->slots[i]);
    if (ctx->d_timing) cudaFree(ctx->d_timing);
    if (ctx->d_progress) cudaFree(ctx->d_progress);
    if (ctx->gemm_ws) cudaFree(ctx->gemm_ws);
    if (ctx->gemm_cnt) cudaFree(ctx->gemm_cnt);
    if (ctx->s_stress) cudaStreamDestroy(ctx->s_stress);
    if (ctx->s_victim) cudaStreamDestroy(ctx->s_victim);
    if (ctx->s_ctrl) cudaStreamDestroy(ctx->s_ctrl);
    if (ctx->h_one) cudaFreeHost(ctx->h_one);
    if (ctx->ev_a) cudaEventDestroy(ctx->ev_a);
    if (ctx->ev_b) cudaEventDestroy(ctx->ev_b);
    free(ctx);
}

extern "C" int ifr_device_query(ifr_ctx *ctx, ifr_device_info *out) {
    if (!ctx || !out) return IFR_ERR_ARG;
    *out = ctx->info;
    return IFR_OK;
}

int ifr_slot_alloc(ifr_ctx *ctx) {
    for (int i = 0; i < IFR_SLOTS; ++i)
        if (!ctx->slots[i].in_use) return i;
    return IFR_ERR_CAPACITY;
}

int ifr_slot_prepare(ifr_ctx *ctx, int slot) {
    Slot &s = ctx->slots[slot];
    if (!s.d_state) {
        IFR_CUDA(cudaMalloc(&s.d_state, sizeof(DevStress)));
        IFR_CUDA(cudaMemset(s.d_state, 0, sizeof(DevStress)));
    }
    int cap = ctx->info.num_sms * IFR_MAX_BPS;
    if (!s.d_logs) {
        IFR_CUDA(cudaMalloc(&s.d_logs, sizeof(ifr_block_log) * (size_t)cap));
        s.log_cap = cap;
        s.h_logs = (ifr_block_log *)calloc((size_t)cap, sizeof(ifr_block_log));
        if (!s.h_logs) return IFR_ERR_NOMEM;
    }
    if (!s.ev_start) {
        IFR_CUDA(cudaEventCreate(&s.ev_start));
        IFR_CUDA(cudaEventCreate(&s.ev_end));
        IFR_CUDA(cudaEventCreateWithFlags(&s.ev_reset, cudaEventDisableTiming));
    }
    return IFR_OK;
}

int ifr_preload(const void *func) {
    cudaFuncAttributes a;
    IFR_CUDA(cudaFuncGetAttributes(&a, func));
    ifr_carveout(func);
    return IFR_OK;
}

void ifr_carveout(const void *func) {
    static std::mutex mu;
    static std::unordered_set<const void *> done;
    std::lock_guard<std::mutex> g(mu);
    if (done.insert(func).second)
        cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

// SMs allowed for a stressor using sm_count of num_sms SMs: spread evenly over
// the SM id range (SM s is allowed when floor((s+1)f) > floor(s f), f = count/num).
void ifr_compute_mask(int num_sms, int sm_count, uint32_t *mask) {
    for (int i = 0; i < IFR_MAX_SMS / 32; ++i) mask[i] = 0u;
    if (sm_count <= 0) return;
    if (sm_count > num_sms) sm_count = num_sms;
    for (int s = 0; s < num_sms; ++s) {
        long long a = (long long)(s + 1) * sm_count / num_sms;
        long long b = (long long)s * sm_count / num_sms;
        if (a > b) mask[s >> 5] |= 1u << (s & 31);
    }
}
