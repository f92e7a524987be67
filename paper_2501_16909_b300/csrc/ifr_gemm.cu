// BF16 GEMM victim on the 5th-generation tensor cores: C[m][n] = sum_k A[m][k] B[n][k]
// (A is M x K and B is N x K, both row-major bf16, i.e. K-major operands; C fp32).
// The paper's shared-memory experiment colocates torch.mm (cuBLAS) with a strided
// shared-memory stressor (Sec. 4.4.1); this is the library's own GEMM.
//
// One CTA computes a 128 x BN tile (BN = 256, or 128 when N is not a multiple of
// 256) with 192 threads:
//   warp 0, lane 0   TMA producer: 64-wide K slices of A (128 rows) and B (BN rows)
//                    into a STAGES-deep ring of 128-byte-swizzled shared tiles
//   warp 1           allocates BN TMEM columns; lane 0 issues tcgen05.mma
//                    (M = 128, N = BN, K = 16) and commits each stage back to the
//                    producer, then the finished accumulator to the epilogue
//   warps 2..5       epilogue: TMEM -> registers (tcgen05.ld) -> fp32 C rows
// Every mbarrier wait is bounded; a CTA that times out records IFR_ERR_TIMEOUT in
// the measurement's status, drains its outstanding TMA copies and frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "ifr_internal.cuh"
#include "ifr_tcgen05.cuh"

namespace {

// Three stages (147 KiB of shared memory at BN = 256) leave room on the SM for a
// stressor block (the tensor stressor needs 34 KiB, the shared-memory stressor
// 2 x 33 KiB): a colocation-friendly configuration in the sense of Sec. 5.3.
// Four stages (195 KiB) would make the GEMM and those stressors mutually exclusive.
constexpr int BM = 128, BK = 64, STAGES = 3;
constexpr uint64_t kGemmTimeoutNs = 1000000000ull;

template <int BN>
struct GemmCfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
};

__device__ __forceinline__ void g_enter(DevTiming *tm) {
    if (threadIdx.x == 0) {
        const unsigned long long t = ifr_gtimer();
        atomicMin((unsigned long long *)&tm->t_min, t);
        if (tm->progress) atomicMax((unsigned long long *)tm->progress, t);
    }
}
__device__ __forceinline__ void g_exit(DevTiming *tm) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t = ifr_gtimer();
        atomicMax((unsigned long long *)&tm->t_max, t);
        if (tm->progress) atomicMax((unsigned long long *)tm->progress, t);
        atomicAdd(&tm->blocks, 1u);
        const uint32_t s = ifr_smid();
        if (s < IFR_MAX_SMS) atomicOr(&tm->sm_bits[s >> 5], 1u << (s & 31));
    }
}

template <int BN>
__global__ void __launch_bounds__(192, 1) gemm_bf16_kernel(const __grid_constant__ CUtensorMap ta,
                                                           const __grid_constant__ CUtensorMap tb,
                                                           float *__restrict__ C, int N, int K, DevTiming *tm) {
    using Cf = GemmCfg<BN>;
    extern __shared__ uint8_t g_smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)g_smem_raw + 1023u) & ~(uintptr_t)1023u);
    uint64_t *full = (uint64_t *)(base + STAGES * Cf::STAGE);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint32_t *tmem_slot = (uint32_t *)(tfull + 1);
    volatile int *fail = (volatile int *)(tmem_slot + 1);

    g_enter(tm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int KT = K / BK;
    const uint64_t deadline = ifr_gtimer() + kGemmTimeoutNs;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(tfull, 1);
        *fail = 0;
        tc::fence_mbar_init();
        tc::prefetch_tmap(&ta);
        tc::prefetch_tmap(&tb);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, BN);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int kt = 0; kt < KT; ++kt) {
            const int s = kt % STAGES;
            if (kt >= STAGES && !tc::mbar_wait(&empty[s], (uint32_t)((kt / STAGES) - 1) & 1u, deadline)) {
                *fail = 1;
                break;
            }
            uint8_t *sa = base + s * Cf::STAGE;
            tc::mbar_arrive_expect_tx(&full[s], (uint32_t)Cf::STAGE);
            tc::tma_load_2d(sa, &ta, &full[s], kt * BK, m0);
            tc::tma_load_2d(sa + Cf::A_BYTES, &tb, &full[s], kt * BK, n0);
            issued = kt + 1;
        }
        // drain: the copies of the last stages have landed before the CTA may exit
        for (int kt = issued - STAGES < 0 ? 0 : issued - STAGES; kt < issued; ++kt)
            tc::mbar_wait(&full[kt % STAGES], (uint32_t)(kt / STAGES) & 1u, deadline + 100000000ull);
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
        for (int kt = 0; kt < KT; ++kt) {
            const int s = kt % STAGES;
            if (!tc::mbar_wait(&full[s], (uint32_t)(kt / STAGES) & 1u, deadline)) {
                *fail = 1;
                break;
            }
            tc::fence_after();
            const uint32_t sa = tc::smem_u32(base + s * Cf::STAGE);
            const uint64_t adesc = tc::desc_sw128(sa);
            const uint64_t bdesc = tc::desc_sw128(sa + Cf::A_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                tc::mma_bf16(tmem, adesc + 2ull * kk, bdesc + 2ull * kk, idesc, (uint32_t)((kt | kk) != 0));
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(tfull);
    } else if (warp >= 2) {
        const int q = warp & 3;  // TMEM lane quadrant this warp may access
        const bool ok = tc::mbar_wait(tfull, 0u, deadline + 100000000ull);
        tc::fence_after();
        if (__all_sync(0xffffffffu, ok && !*fail)) {
            float *crow = C + (size_t)(m0 + q * 32 + lane) * (size_t)N + n0;
#pragma unroll 1
            for (int cc = 0; cc < BN; cc += 32) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cc, r);
                tc::tmem_ld_wait();
                float4 *dst = (float4 *)(crow + cc);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                         __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
            }
        } else if (lane == 0) {
            *fail = 1;
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, BN);
    }
    if (threadIdx.x == 0 && *fail) tm->status = IFR_ERR_TIMEOUT;
    g_exit(tm);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D map over a rows x K bf16 row-major matrix, box = 64 (K) x box_rows, 128-B swizzle.
int make_map(CUtensorMap *m, const void *ptr, int64_t rows, int64_t K, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return IFR_ERR_UNSUPPORTED;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? IFR_OK : IFR_ERR_ARG;
}

template <int BN>
int launch_gemm(const ifr_victim_cfg *c, cudaStream_t stream, DevTiming *tm) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gemm_bf16_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, GemmCfg<BN>::SMEM);
        attr = true;
    }
    CUtensorMap ta, tb;
    int rc = make_map(&ta, c->in0, c->m, c->k, BM);
    if (rc) return rc;
    rc = make_map(&tb, c->in1, c->n, c->k, BN);
    if (rc) return rc;
    ifr_carveout((const void *)gemm_bf16_kernel<BN>);
    dim3 grid((unsigned)(c->n / BN), (unsigned)(c->m / BM));
    gemm_bf16_kernel<BN><<<grid, 192, GemmCfg<BN>::SMEM, stream>>>(ta, tb, (float *)c->out, (int)c->n, (int)c->k, tm);
    return IFR_OK;
}

}  // namespace

int ifr_gemm_shape(const ifr_victim_cfg *c, VictimShape *s) {
    const bool wide = c->n % 256 == 0;
    s->fn = wide ? (const void *)gemm_bf16_kernel<256> : (const void *)gemm_bf16_kernel<128>;
    s->grid = (int)((c->n / (wide ? 256 : 128)) * (c->m / BM));
    s->block = 192;
    s->smem = wide ? GemmCfg<256>::SMEM : GemmCfg<128>::SMEM;
    s->tmem_cols = wide ? 256 : 128;
    s->uses_tensor = 1;
    s->flops = 2.0 * (double)c->m * (double)c->n * (double)c->k;
    s->bytes = 2.0 * ((double)c->m + (double)c->n) * (double)c->k + 4.0 * (double)c->m * (double)c->n;
    return IFR_OK;
}

int ifr_gemm_enqueue(ifr_ctx *, const ifr_victim_cfg *c, cudaStream_t stream, DevTiming *tm) {
    if (c->m > 65535 * BM || c->n > (1ll << 30) || c->k > (1ll << 30)) return IFR_ERR_ARG;
    if (c->n % 256 == 0) return launch_gemm<256>(c, stream, tm);
    return launch_gemm<128>(c, stream, tm);
}
