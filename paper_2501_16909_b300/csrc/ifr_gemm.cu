// BF16 GEMM victim on the 5th-generation tensor cores: C[m][n] = sum_k A[m][k] B[n][k]
// (A is M x K and B is N x K, both row-major bf16, i.e. K-major operands; C fp32).
// The paper's shared-memory experiment colocates torch.mm (cuBLAS) with a strided
// shared-memory stressor (Sec. 4.4.1); this is the library's own GEMM.
//
// Persistent: one CTA per SM takes 128 x BN output tiles (BN = 256, or 128 when N is
// not a multiple of 256) until none are left: its first tile is its own index, every
// later one comes from a device counter (tile order: see tile_coords).  Handing tiles
// out on demand keeps the load balance of a one-CTA-per-tile launch: a CTA on an SM
// that a stressor slows takes fewer tiles instead of holding up the grid with a fixed
// share.  A second kernel below runs 256 x 256 tiles on CTA pairs.  192 threads:
//   warp 0, lane 0   tile scheduler and TMA producer: takes tile blockIdx.x first and
//                    then claims tiles gridDim.x, gridDim.x + 1, ... from the counter; publishes
//                    its index in a 4-entry shared ring for the other roles, and loads
//                    64-wide K slices of A (128 rows) and B (BN rows)
//                    into a STAGES-deep ring of 128-byte-swizzled shared tiles; the
//                    ring runs on across tile boundaries, so the next tile's loads
//                    overlap the current tile's epilogue
//   warp 1           allocates BN TMEM columns (one fp32 accumulator); lane 0 issues
//                    tcgen05.mma (M = 128, N = BN, K = 16), commits every stage back to
//                    the producer and every finished tile to the epilogue
//   warps 2..5       epilogue, one warp per TMEM lane quadrant: 16-column chunks are
//                    read with tcgen05.ld while the previous chunk is stored to C; the
//                    accumulator is released after the last chunk's read
// Registers are granted per SM sub-partition (four 16 K files, the block's warps
// spread over them), so beside the widest stressor pair (2 x 512 threads x 40
// registers: 8 warps x 1280 on every sub-partition) two GEMM warps must fit in 6144
// registers: at most 96 per thread, which the 16-column chunks keep.
// Every mbarrier wait is bounded; a CTA that times out records IFR_ERR_TIMEOUT in
// the measurement's status, drains its outstanding TMA copies and frees TMEM.  The
// last CTA of a launch to finish returns the tile counter to zero for the next one
// (launches on one measurement record are stream-ordered).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "ifr_internal.cuh"
#include "ifr_tcgen05.cuh"

namespace {

// Variants 0 and 1 (Sec. 5.3: colocation-friendly kernel variants; variant 2, the
// CTA-pair kernel, is described with it).  Three stages (145 KiB
// of shared memory at BN = 256) leave room on the SM for a stressor block (the tensor
// stressor needs 34 KiB, the shared-memory stressor 2 x 33 KiB).  Four stages
// (193 KiB) keep a third more operand bytes in flight, which the single-CTA tile needs
// to cover the L2 round trip, but make the GEMM and those stressors mutually
// exclusive on an SM.  One BN-column accumulator (not two) leaves TMEM for the tensor
// stressor in both.
constexpr int BM = 128, BK = 64, EPI_WARPS = 4, GEMM_THREADS = 64 + 32 * EPI_WARPS;
constexpr int RING = 4;  // tile indices in flight between the scheduler and the consumers
constexpr uint64_t kGemmTimeoutNs = 4000000000ull;
int g_num_sms = 0;  // persistent grid size (set from the context before each launch)

// Work split of one launch (variant 3).  Units 0 .. full-1 are whole tiles (unit =
// tile).  When the tiles do not fill the last wave of CTAs, the tiles after `full`
// are computed as `parts` K ranges each, units full + t*parts + part, so that the
// last wave holds parts x as many, shorter units.  Each part stores its partial
// tile in its slot of `ws`; per (tile, epilogue warp) a counter counts the parts
// that have stored (modulo parts, so it needs no reset between launches), and the
// last to arrive adds the slots in part order and stores C.  parts = 1: no split.
struct GemmSplit {
    int full;
    int parts;
    float *ws;      // [split tiles][parts][BM][BN] fp32 partial tiles
    uint32_t *cnt;  // [split tiles][EPI_WARPS] arrival counters
};

template <bool SPLIT>
__device__ __forceinline__ void unit_of(int u, const GemmSplit &sp, int KT, int &tile, int &k0, int &k1, int &part,
                                        int &fix) {
    if (!SPLIT || sp.parts <= 1 || u < sp.full) {
        tile = u;
        k0 = 0;
        k1 = KT;
        part = 0;
        fix = -1;
    } else {
        const int v = u - sp.full;
        fix = v / sp.parts;
        part = v % sp.parts;
        tile = sp.full + fix;
        k0 = part * KT / sp.parts;
        k1 = (part + 1) * KT / sp.parts;
    }
}

template <int BN, int STAGES>
struct GemmCfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;  // + alignment slack + barriers / ring
};

__device__ __forceinline__ void g_stamp(DevTiming *tm, bool first) {
    const unsigned long long t = ifr_gtimer();
    if (first) atomicMin((unsigned long long *)&tm->t_min, t);
    if (tm->progress) atomicMax((unsigned long long *)tm->progress, t);
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

// Tile index -> (tile row, tile column) in groups of `group_m` tile rows: consecutive
// tiles walk down a group's rows before moving one tile column right, so the tiles in
// flight at once share a few A and B panels in L2 instead of sweeping every B panel
// while they share one A panel.  group_m = 1 is row-major order, which the launch
// keeps when A and B fit in L2 together (measured at 4096^3: grouping there read 20 %
// more DRAM bytes).  Every tile is still computed the same way; only the order in
// which tiles are handed out changes.
constexpr int GROUP_M = 8;
__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int group_m, int &tm, int &tn) {
    const int per_group = group_m * tiles_n;
    const int first_m = (tile / per_group) * group_m;
    const int rows = tiles_m - first_m < group_m ? tiles_m - first_m : group_m;
    const int in_group = tile % per_group;
    tm = first_m + in_group % rows;
    tn = in_group / rows;
}

// 16 consecutive fp32 values of one C row (64 B) as four 16-byte stores.
__device__ __forceinline__ void store_row16(float *dst, const uint32_t (&r)[16]) {
    float4 *d = (float4 *)dst;
#pragma unroll
    for (int e = 0; e < 4; ++e)
        d[e] = make_float4(__uint_as_float(r[4 * e]), __uint_as_float(r[4 * e + 1]), __uint_as_float(r[4 * e + 2]),
                           __uint_as_float(r[4 * e + 3]));
}

// One epilogue warp's 32 rows of a split tile are in this part's slot: count the
// part on the (tile, warp) counter; the last part to arrive adds the 32 rows of every
// slot in part order and stores them to C.  Coalesced: the warp walks its rows four
// at a time with the lanes across the columns (BN / 128 float4 per lane per row), the
// loads of the four rows of all parts in flight together.  slot0: row 0 of part 0;
// part_stride: floats from one part's slot to the next.
template <int BN>
__device__ __forceinline__ void split_arrive_reduce(const GemmSplit &sp, uint32_t *cnt, const float *slot0,
                                                    size_t part_stride, float *cq, int N, int lane) {
    __threadfence();
    __syncwarp();
    uint32_t prev = 0;
    if (lane == 0) prev = atomicAdd(cnt, 1u);
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if ((prev + 1u) % (uint32_t)sp.parts != 0u) return;
    __threadfence();
    constexpr int H = BN / 128;
#pragma unroll 1
    for (int r0 = 0; r0 < 32; r0 += 4) {
        float4 t[4][H];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int h = 0; h < H; ++h) t[rr][h] = __ldcg((const float4 *)(slot0 + (size_t)(r0 + rr) * BN) + lane + 32 * h);
#pragma unroll 1
        for (int pp = 1; pp < sp.parts; ++pp) {
            const float *sl = slot0 + (size_t)pp * part_stride;
            float4 u[4][H];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int h = 0; h < H; ++h) u[rr][h] = __ldcg((const float4 *)(sl + (size_t)(r0 + rr) * BN) + lane + 32 * h);
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    t[rr][h].x += u[rr][h].x;
                    t[rr][h].y += u[rr][h].y;
                    t[rr][h].z += u[rr][h].z;
                    t[rr][h].w += u[rr][h].w;
                }
        }
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int h = 0; h < H; ++h) ((float4 *)(cq + (size_t)(r0 + rr) * N))[lane + 32 * h] = t[rr][h];
    }
}

// ACC accumulators of BN TMEM columns: with two, the MMAs of the next unit run into
// one while the epilogue drains the other (variant 3, for solo use: 512 columns
// leave no TMEM for other kernels on the SM).  SPLIT compiles the split last wave
// in (variant 3 only: the other variants keep their registers).
template <int BN, int STAGES, int ACC, bool SPLIT>
__global__ void __launch_bounds__(GEMM_THREADS, 1) gemm_bf16_kernel(const __grid_constant__ CUtensorMap ta,
                                                                    const __grid_constant__ CUtensorMap tb,
                                                                    float *__restrict__ C, int M, int N, int K,
                                                                    int group_m, GemmSplit sp, DevTiming *tm) {
    using Cf = GemmCfg<BN, STAGES>;
    constexpr int CHUNKS = BN / 16;
    extern __shared__ uint8_t g_smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)g_smem_raw + 1023u) & ~(uintptr_t)1023u);
    uint64_t *full = (uint64_t *)(base + STAGES * Cf::STAGE);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;  // [ACC]
    uint64_t *tempty = tfull + ACC;    // [ACC]
    uint64_t *sfull = tempty + ACC;    // [RING] unit index published
    uint64_t *sempty = sfull + RING;   // [RING] unit index read by the MMA lane and 4 epilogue warps
    int32_t *ring = (int32_t *)(sempty + RING);
    uint32_t *tmem_slot = (uint32_t *)(ring + RING);
    volatile int *fail = (volatile int *)(tmem_slot + 1);

    if (threadIdx.x == 0) g_stamp(tm, true);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = M / BM, tiles_n = N / BN, n_tiles = tiles_m * tiles_n;
    const int KT = K / BK;
    const int n_units = (SPLIT && sp.parts > 1) ? sp.full + (n_tiles - sp.full) * sp.parts : n_tiles;
    const uint64_t deadline = ifr_gtimer() + kGemmTimeoutNs;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int r = 0; r < RING; ++r) {
            tc::mbar_init(&sfull[r], 1);
            tc::mbar_init(&sempty[r], 1 + EPI_WARPS);
        }
        for (int a = 0; a < ACC; ++a) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], EPI_WARPS);
        }
        *fail = 0;
        tc::fence_mbar_init();
        tc::prefetch_tmap(&ta);
        tc::prefetch_tmap(&tb);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, ACC * BN);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        int64_t g = 0;
        // The following tile is claimed just before the wait for the current tile's
        // last free stage, so the atomic's round trip hides behind that wait while the
        // CTA holds the claim only for the stages still in flight.
        uint32_t next = blockIdx.x;  // first tile: the CTA's own index; later ones from the counter
        for (int j = 0;; ++j) {
            const int r = j % RING;
            if (j >= RING && !tc::mbar_wait(&sempty[r], (uint32_t)((j / RING) - 1) & 1u, deadline)) *fail = 1;
            const int unit = (*fail || next >= (uint32_t)n_units) ? -1 : (int)next;
            ring[r] = unit;
            tc::mbar_arrive(&sfull[r]);  // release: the index is visible to the waiting roles
            if (unit < 0) break;
            int tile, k0, k1, part, fix;
            unit_of<SPLIT>(unit, sp, KT, tile, k0, k1, part, fix);
            int tmi, tni;
            tile_coords(tile, tiles_m, tiles_n, group_m, tmi, tni);
            const int m0 = tmi * BM, n0 = tni * BN;
            for (int kt = k0; kt < k1; ++kt, ++g) {
                const int s = (int)(g % STAGES);
                if (kt == k1 - 1) next = gridDim.x + atomicAdd(&tm->tile_next, 1u);
                if (g >= STAGES && !tc::mbar_wait(&empty[s], (uint32_t)((g / STAGES) - 1) & 1u, deadline)) {
                    *fail = 1;
                    break;
                }
                uint8_t *sa = base + s * Cf::STAGE;
                tc::mbar_arrive_expect_tx(&full[s], (uint32_t)Cf::STAGE);
                tc::tma_load_2d(sa, &ta, &full[s], kt * BK, m0);
                tc::tma_load_2d(sa + Cf::A_BYTES, &tb, &full[s], kt * BK, n0);
            }
        }
        // drain: the copies of the last stages have landed before the CTA may exit
        for (int64_t q = g - STAGES < 0 ? 0 : g - STAGES; q < g; ++q)
            tc::mbar_wait(&full[q % STAGES], (uint32_t)(q / STAGES) & 1u, deadline + 100000000ull);
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
        int64_t g = 0;
        for (int j = 0;; ++j) {
            const int r = j % RING;
            const bool got = tc::mbar_wait(&sfull[r], (uint32_t)(j / RING) & 1u, deadline + 50000000ull);
            const int unit = got ? ring[r] : -1;
            tc::mbar_arrive(&sempty[r]);
            if (!got) *fail = 1;
            if (unit < 0) break;
            int tile, k0, k1, part, fix;
            unit_of<SPLIT>(unit, sp, KT, tile, k0, k1, part, fix);
            const int a = j % ACC;  // accumulator of this unit
            if (j >= ACC && !tc::mbar_wait(&tempty[a], (uint32_t)((j / ACC) - 1) & 1u, deadline)) {
                *fail = 1;
                tc::mma_commit(&tfull[a]);
                continue;  // read the ring on to its end marker
            }
            tc::fence_after();
            const uint32_t acc_cols = tmem + (uint32_t)(a * BN);
            for (int kt = k0; kt < k1; ++kt, ++g) {
                const int s = (int)(g % STAGES);
                if (!tc::mbar_wait(&full[s], (uint32_t)(g / STAGES) & 1u, deadline)) {
                    *fail = 1;
                    break;
                }
                tc::fence_after();
                const uint32_t sa = tc::smem_u32(base + s * Cf::STAGE);
                const uint64_t adesc = tc::desc_sw128(sa);
                const uint64_t bdesc = tc::desc_sw128(sa + Cf::A_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    tc::mma_bf16(acc_cols, adesc + 2ull * kk, bdesc + 2ull * kk, idesc,
                                 (uint32_t)((kt != k0) | (kk != 0)));
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(&tfull[a]);  // also on failure, so the epilogue's wait completes
        }
    } else if (warp >= 2) {
        const int q = warp & 3;  // TMEM lane quadrant this warp may access
        for (int j = 0;; ++j) {
            const int r = j % RING;
            const bool got = tc::mbar_wait(&sfull[r], (uint32_t)(j / RING) & 1u, deadline + 50000000ull);
            const int unit = got ? ring[r] : -1;
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sempty[r]);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) *fail = 1;
                break;
            }
            if (unit < 0) break;
            const int a = j % ACC;
            const bool ok = tc::mbar_wait(&tfull[a], (uint32_t)(j / ACC) & 1u, deadline + 100000000ull);
            tc::fence_after();
            if (!__all_sync(0xffffffffu, ok && !*fail)) {
                if (lane == 0) *fail = 1;
                break;
            }
            int tile, k0, k1, part, fix;
            unit_of<SPLIT>(unit, sp, KT, tile, k0, k1, part, fix);
            const uint32_t trow = tmem + (uint32_t)(a * BN) + ((uint32_t)(q * 32) << 16);
            int tmi, tni;
            tile_coords(tile, tiles_m, tiles_n, group_m, tmi, tni);
            const int m0 = tmi * BM, n0 = tni * BN;
            // a whole tile's rows go to C; a part's rows go to its slot of the workspace
            float *crow = (!SPLIT || fix < 0) ? C + (size_t)(m0 + q * 32 + lane) * (size_t)N + n0
                                  : sp.ws + ((size_t)(fix * sp.parts + part) * BM + (size_t)(q * 32 + lane)) * BN;
            uint32_t ra[16], rb[16];
            tc::tmem_ld16(trow, ra);
            tc::tmem_ld_wait();
#pragma unroll
            for (int c = 0; c < CHUNKS; c += 2) {
                tc::tmem_ld16(trow + (uint32_t)((c + 1) * 16), rb);
                store_row16(crow + c * 16, ra);
                tc::tmem_ld_wait();
                if (c + 2 < CHUNKS) {
                    tc::tmem_ld16(trow + (uint32_t)((c + 2) * 16), ra);
                    store_row16(crow + (c + 1) * 16, rb);
                    tc::tmem_ld_wait();
                } else {
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&tempty[a]);  // accumulator drained: a later unit may use it
                    store_row16(crow + (c + 1) * 16, rb);
                }
            }
            if (SPLIT && fix >= 0)
                split_arrive_reduce<BN>(sp, &sp.cnt[fix * EPI_WARPS + q],
                                        sp.ws + ((size_t)fix * sp.parts * BM + (size_t)(q * 32)) * BN,
                                        (size_t)BM * BN, C + (size_t)(m0 + q * 32) * (size_t)N + n0, N, lane);
            if (warp == 2 && lane == 0) g_stamp(tm, false);  // victim progress, one stamp per unit
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, ACC * BN);
    }
    if (threadIdx.x == 0 && *fail) tm->status = IFR_ERR_TIMEOUT;
    g_exit(tm);
    if (threadIdx.x == 0) {
        // every CTA has claimed its last tile before it counts itself done
        __threadfence();
        if (atomicAdd(&tm->tile_done, 1u) == gridDim.x - 1u) {
            atomicExch(&tm->tile_next, 0u);
            atomicExch(&tm->tile_done, 0u);
        }
    }
}

// ------------------------------------------------------------------ grouped GEMM
// The grouped victims of a graph-batched sweep: up to IFR_GROUP_MAX GEMMs of
// one tile width run as one persistent launch of variant 0's tiles (three stages, one
// accumulator).  Units are the concatenation of the problems' tiles in order
// (problem q owns units tile0[q] ..), every unit claimed from the device counter of
// problem 0's record.  A producer that takes its first tile of problem q waits until
// every tile of problem q - 1 is stored (the four epilogue warps of each tile count
// themselves in problem q - 1's record), so the problems still run one after
// another, as separate launches would, without the launch gaps; the wait cannot
// deadlock, since every tile of an earlier problem was claimed before, by a running
// CTA.  Each problem keeps its own measurement record: the producer stamps entry at a
// tile's first K slice (after the wait) and each epilogue warp stamps exit at the
// tile's end, so a problem's span runs from its first tile's start to its last tile's
// end.  Waits are bounded as in the single kernel; a CTA that times out records
// IFR_ERR_TIMEOUT in every problem's record.
struct alignas(64) GemmProblem {
    CUtensorMap ta, tb;
    float *C;
    DevTiming *tm;
    int32_t N, K, tiles_m, tiles_n, tile0, group_m;
};
struct GemmGroup {
    GemmProblem p[IFR_GROUP_MAX];
    int32_t n, total;
};

__device__ __forceinline__ int group_problem(const GemmGroup &g, int u) {
    int q = 0;
    while (q + 1 < g.n && u >= g.p[q + 1].tile0) ++q;
    return q;
}

// Bounded wait (the producer thread) until every tile of problem q - 1 is stored.
__device__ __forceinline__ bool group_wait_tiles(const GemmGroup &g, int q, uint64_t deadline) {
    if (q == 0) return true;
    const GemmProblem &pp = g.p[q - 1];
    const uint32_t want = (uint32_t)(EPI_WARPS * pp.tiles_m * pp.tiles_n);
    uint32_t it = 0;
    while (*(const volatile uint32_t *)&pp.tm->done < want) {
        if (ifr_gtimer() > deadline || ++it > (1u << 24)) return false;
        __nanosleep(200);
    }
    __threadfence();
    return true;
}

__device__ __forceinline__ void g_tile_exit(DevTiming *tm, bool count) {
    const unsigned long long t = ifr_gtimer();
    atomicMax((unsigned long long *)&tm->t_max, t);
    if (tm->progress) atomicMax((unsigned long long *)tm->progress, t);
    if (count) {
        atomicAdd(&tm->blocks, 1u);
        const uint32_t s = ifr_smid();
        if (s < IFR_MAX_SMS) atomicOr(&tm->sm_bits[s >> 5], 1u << (s & 31));
    }
}

template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1) gemm_bf16_group_kernel(const __grid_constant__ GemmGroup g) {
    constexpr int STAGES = 3;
    using Cf = GemmCfg<BN, STAGES>;
    constexpr int CHUNKS = BN / 16;
    extern __shared__ uint8_t g_smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)g_smem_raw + 1023u) & ~(uintptr_t)1023u);
    uint64_t *full = (uint64_t *)(base + STAGES * Cf::STAGE);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + 1;
    uint64_t *sfull = tempty + 1;   // [RING] unit index published
    uint64_t *sempty = sfull + RING;  // [RING] unit index read by the MMA lane and 4 epilogue warps
    int32_t *ring = (int32_t *)(sempty + RING);
    uint32_t *tmem_slot = (uint32_t *)(ring + RING);
    volatile int *fail = (volatile int *)(tmem_slot + 1);
    DevTiming *const ctl = g.p[0].tm;  // holds the unit counter

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t deadline = ifr_gtimer() + kGemmTimeoutNs;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int r = 0; r < RING; ++r) {
            tc::mbar_init(&sfull[r], 1);
            tc::mbar_init(&sempty[r], 1 + EPI_WARPS);
        }
        tc::mbar_init(tfull, 1);
        tc::mbar_init(tempty, EPI_WARPS);
        *fail = 0;
        tc::fence_mbar_init();
        for (int q = 0; q < g.n; ++q) {
            tc::prefetch_tmap(&g.p[q].ta);
            tc::prefetch_tmap(&g.p[q].tb);
        }
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
        int64_t gs = 0;
        uint32_t next = atomicAdd(&ctl->tile_next, 1u);
        int waited = 0;  // problems before `waited` are known finished
        for (int j = 0;; ++j) {
            const int r = j % RING;
            if (j >= RING && !tc::mbar_wait(&sempty[r], (uint32_t)((j / RING) - 1) & 1u, deadline)) *fail = 1;
            const int unit = (*fail || next >= (uint32_t)g.total) ? -1 : (int)next;
            ring[r] = unit;
            tc::mbar_arrive(&sfull[r]);
            if (unit < 0) break;
            const int q = group_problem(g, unit);
            const GemmProblem &pb = g.p[q];
            if (q > waited) {
                if (!group_wait_tiles(g, q, deadline)) *fail = 1;
                waited = q;
            }
            int tmi, tni;
            tile_coords(unit - pb.tile0, pb.tiles_m, pb.tiles_n, pb.group_m, tmi, tni);
            const int m0 = tmi * BM, n0 = tni * BN, KT = pb.K / BK;
            g_stamp(pb.tm, true);
            for (int kt = 0; kt < KT; ++kt, ++gs) {
                const int s = (int)(gs % STAGES);
                if (kt == KT - 1) next = atomicAdd(&ctl->tile_next, 1u);
                if (gs >= STAGES && !tc::mbar_wait(&empty[s], (uint32_t)((gs / STAGES) - 1) & 1u, deadline)) {
                    *fail = 1;
                    break;
                }
                uint8_t *sa = base + s * Cf::STAGE;
                tc::mbar_arrive_expect_tx(&full[s], (uint32_t)Cf::STAGE);
                tc::tma_load_2d(sa, &pb.ta, &full[s], kt * BK, m0);
                tc::tma_load_2d(sa + Cf::A_BYTES, &pb.tb, &full[s], kt * BK, n0);
            }
        }
        // drain: the copies of the last stages have landed before the CTA may exit
        for (int64_t q = gs - STAGES < 0 ? 0 : gs - STAGES; q < gs; ++q)
            tc::mbar_wait(&full[q % STAGES], (uint32_t)(q / STAGES) & 1u, deadline + 100000000ull);
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
        int64_t gs = 0;
        for (int j = 0;; ++j) {
            const int r = j % RING;
            const bool got = tc::mbar_wait(&sfull[r], (uint32_t)(j / RING) & 1u, deadline + 50000000ull);
            const int unit = got ? ring[r] : -1;
            tc::mbar_arrive(&sempty[r]);
            if (!got) *fail = 1;
            if (unit < 0) break;
            const int KT = g.p[group_problem(g, unit)].K / BK;
            if (j >= 1 && !tc::mbar_wait(tempty, (uint32_t)((j - 1) & 1), deadline)) {
                *fail = 1;
                tc::mma_commit(tfull);
                continue;  // read the ring on to its end marker
            }
            tc::fence_after();
            for (int kt = 0; kt < KT; ++kt, ++gs) {
                const int s = (int)(gs % STAGES);
                if (!tc::mbar_wait(&full[s], (uint32_t)(gs / STAGES) & 1u, deadline)) {
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
            tc::mma_commit(tfull);  // also on failure, so the epilogue's wait completes
        }
    } else if (warp >= 2) {
        const int qd = warp & 3;  // TMEM lane quadrant this warp may access
        const uint32_t trow = tmem + ((uint32_t)(qd * 32) << 16);
        for (int j = 0;; ++j) {
            const int r = j % RING;
            const bool got = tc::mbar_wait(&sfull[r], (uint32_t)(j / RING) & 1u, deadline + 50000000ull);
            const int unit = got ? ring[r] : -1;
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sempty[r]);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) *fail = 1;
                break;
            }
            if (unit < 0) break;
            const bool ok = tc::mbar_wait(tfull, (uint32_t)(j & 1), deadline + 100000000ull);
            tc::fence_after();
            if (!__all_sync(0xffffffffu, ok && !*fail)) {
                if (lane == 0) *fail = 1;
                break;
            }
            const GemmProblem &pb = g.p[group_problem(g, unit)];
            int tmi, tni;
            tile_coords(unit - pb.tile0, pb.tiles_m, pb.tiles_n, pb.group_m, tmi, tni);
            const int m0 = tmi * BM, n0 = tni * BN;
            float *crow = pb.C + (size_t)(m0 + qd * 32 + lane) * (size_t)pb.N + n0;
            uint32_t ra[16], rb[16];
            tc::tmem_ld16(trow, ra);
            tc::tmem_ld_wait();
#pragma unroll
            for (int c = 0; c < CHUNKS; c += 2) {
                tc::tmem_ld16(trow + (uint32_t)((c + 1) * 16), rb);
                store_row16(crow + c * 16, ra);
                tc::tmem_ld_wait();
                if (c + 2 < CHUNKS) {
                    tc::tmem_ld16(trow + (uint32_t)((c + 2) * 16), ra);
                    store_row16(crow + (c + 1) * 16, rb);
                    tc::tmem_ld_wait();
                } else {
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(tempty);  // accumulator drained
                    store_row16(crow + (c + 1) * 16, rb);
                }
            }
            // every epilogue warp stamps the tile's end (the latest of the four is the
            // tile's exit) and counts itself for the ordering of the next problem;
            // warp 2 also counts the tile and its SM
            __syncwarp();
            if (lane == 0) {
                g_tile_exit(pb.tm, warp == 2);
                __threadfence();
                atomicAdd(&pb.tm->done, 1u);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, BN);
    }
    if (threadIdx.x == 0 && *fail)
        for (int q = 0; q < g.n; ++q) g.p[q].tm->status = IFR_ERR_TIMEOUT;
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctl->tile_done, 1u) == gridDim.x - 1u) {
            for (int q = 0; q < g.n; ++q) atomicExch(&g.p[q].tm->done, 0u);
            atomicExch(&ctl->tile_next, 0u);
            atomicExch(&ctl->tile_done, 0u);
        }
    }
}

// ------------------------------------------------------------------ 2-SM pair tiles
// Variant 2: a cluster of two CTAs on two SMs takes 256 x 256 output tiles with
// tcgen05.mma.cta_group::2 (M = 256, N = 256, K = 16), issued by the even CTA (the
// leader).  Each CTA loads its own 128 rows of A and its own 128 rows of B per 64-wide
// K slice: 32 KiB per stage per SM where the single-CTA tile needs 48 KiB for the same
// MMA work, so six stages (193 KiB) hold 1.5 times the MMA time in operands that four
// 48 KiB stages hold for the single-CTA tile.  Each CTA keeps its 128 rows of the
// accumulator in its own TMEM columns and stores them.  The paired allocation needs
// the same columns free on both SMs, which other TMEM users of those SMs (a tensor
// stressor) can withhold until they exit, so this variant is not a victim beside them.
// The library runs it with STAGES = 6, ACC = 2 and SPLIT:
//   * two 256-column accumulators per CTA (all 512 columns): the next unit's MMAs run
//     into one while both epilogues drain the other;
//   * the split last wave: units as in the single-CTA kernel, over pair tiles.  Each
//     CTA's epilogue warps store their 32 rows of a part into the part's 256-row slot
//     and count it per (tile, CTA, warp); the last part reduces those rows.
//   warp 0, lane 0   TMA producer in both CTAs; in the leader also the unit
//                    scheduler, which writes each unit index into both CTAs' rings.
//                    Both producers complete their bytes on the leader's stage
//                    barrier, whose one arrival (the leader's) expects both CTAs'
//                    bytes: the other CTA's copies may land first, the pending
//                    arrival keeps the phase open until the leader has posted
//   warp 1           allocates the pair's TMEM (both CTAs); leader lane 0 issues the
//                    MMAs and commits each stage and each finished unit to both CTAs
//   warps 2..5       epilogue of the CTA's own 128 accumulator rows; an accumulator
//                    is reused once both CTAs' epilogues have drained it
// Units are handed out as in the single-CTA kernel (first unit = cluster index, later
// ones from the device counter).  Waits are bounded; a teardown cluster barrier
// keeps each CTA resident until the other has finished touching its shared memory.
constexpr int PAIR_M = 256, PAIR_N = 256, HALF = 128;

template <int STAGES>
struct PairCfg {
    static constexpr int A_BYTES = HALF * BK * 2;
    static constexpr int B_BYTES = HALF * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;  // + alignment slack + barriers / ring
};

template <int STAGES, int ACC, bool SPLIT>
__global__ void __launch_bounds__(GEMM_THREADS, 1) gemm_bf16_pair_kernel(const __grid_constant__ CUtensorMap ta,
                                                                         const __grid_constant__ CUtensorMap tb,
                                                                         float *__restrict__ C, int M, int N,
                                                                         int K, int group_m, GemmSplit sp,
                                                                         DevTiming *tm) {
    using Cf = PairCfg<STAGES>;
    constexpr int CHUNKS = PAIR_N / 16;
    constexpr uint16_t kBoth = 3;
    extern __shared__ uint8_t g_smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)g_smem_raw + 1023u) & ~(uintptr_t)1023u);
    uint64_t *full = (uint64_t *)(base + STAGES * Cf::STAGE);  // [STAGES], used in the leader
    uint64_t *empty = full + STAGES;                            // [STAGES], both CTAs
    uint64_t *tfull = empty + STAGES;                           // [ACC], both CTAs
    uint64_t *tempty = tfull + ACC;                             // [ACC], leader
    uint64_t *sfull = tempty + ACC;                             // [RING], both CTAs
    uint64_t *sempty = sfull + RING;                            // [RING], leader
    int32_t *ring = (int32_t *)(sempty + RING);
    uint32_t *tmem_slot = (uint32_t *)(ring + RING);
    volatile int *fail = (volatile int *)(tmem_slot + 1);

    if (tc::cluster_nctarank() != 2) {  // not launched as CTA pairs: touch nothing shared
        if (threadIdx.x == 0) tm->status = IFR_ERR_LAUNCH;
        return;
    }
    const uint32_t rank = tc::cluster_ctarank();
    const bool leader = rank == 0;
    if (threadIdx.x == 0) g_stamp(tm, true);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = M / PAIR_M, tiles_n = N / PAIR_N, n_tiles = tiles_m * tiles_n;
    const int KT = K / BK;
    const int n_units = (SPLIT && sp.parts > 1) ? sp.full + (n_tiles - sp.full) * sp.parts : n_tiles;
    const uint64_t deadline = ifr_gtimer() + kGemmTimeoutNs;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);   // the leader's expect_tx for both CTAs' bytes
            tc::mbar_init(&empty[s], 1);  // the leader's MMA commit
        }
        for (int r = 0; r < RING; ++r) {
            tc::mbar_init(&sfull[r], 1);
            tc::mbar_init(&sempty[r], 2 * (1 + EPI_WARPS));  // leader MMA + peer producer + 2 x 4 epilogue warps
        }
        for (int a = 0; a < ACC; ++a) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], 2 * EPI_WARPS);
        }
        *fail = 0;
        tc::fence_mbar_init();
        tc::prefetch_tmap(&ta);
        tc::prefetch_tmap(&tb);
    }
    if (warp == 1) {
        tc::tmem_alloc_pair(tmem_slot, ACC * PAIR_N);
        tc::tmem_relinquish_pair();
    }
    tc::fence_before();
    tc::cluster_sync();  // both CTAs' barriers are initialised before any remote arrival
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        int64_t g = 0;
        uint32_t next = blockIdx.x >> 1;  // leader: first unit = cluster index, later ones from the counter
        for (int j = 0;; ++j) {
            const int r = j % RING;
            int unit;
            if (leader) {
                if (j >= RING && !tc::mbar_wait_cluster(&sempty[r], (uint32_t)((j / RING) - 1) & 1u, deadline))
                    *fail = 1;
                unit = (*fail || next >= (uint32_t)n_units) ? -1 : (int)next;
                ring[r] = unit;
                tc::st_remote_s32(tc::mapa(&ring[r], 1), unit);
                tc::mbar_arrive(&sfull[r]);
                tc::mbar_arrive_remote(tc::mapa(&sfull[r], 1));  // release: orders the remote ring store
            } else {
                const bool got = tc::mbar_wait_cluster(&sfull[r], (uint32_t)(j / RING) & 1u, deadline + 50000000ull);
                unit = got ? ring[r] : -1;
                if (!got) *fail = 1;
                tc::mbar_arrive_remote(tc::mapa(&sempty[r], 0));
            }
            if (unit < 0) break;
            int tile, k0, k1, part, fix;
            unit_of<SPLIT>(unit, sp, KT, tile, k0, k1, part, fix);
            int tmi, tni;
            tile_coords(tile, tiles_m, tiles_n, group_m, tmi, tni);
            const int m0 = tmi * PAIR_M + (int)rank * HALF, n0 = tni * PAIR_N + (int)rank * HALF;
            for (int kt = k0; kt < k1; ++kt, ++g) {
                const int s = (int)(g % STAGES);
                if (leader && kt == k1 - 1) next = (gridDim.x >> 1) + atomicAdd(&tm->tile_next, 1u);
                if (g >= STAGES && !tc::mbar_wait(&empty[s], (uint32_t)((g / STAGES) - 1) & 1u, deadline)) {
                    *fail = 1;
                    break;
                }
                uint8_t *sa = base + s * Cf::STAGE;
                const uint32_t fb = tc::mapa(&full[s], 0);
                if (leader) tc::mbar_arrive_expect_tx(&full[s], 2u * (uint32_t)Cf::STAGE);
                tc::tma_load_2d_pair(sa, &ta, fb, kt * BK, m0);
                tc::tma_load_2d_pair(sa + Cf::A_BYTES, &tb, fb, kt * BK, n0);
            }
        }
        // the leader's MMAs have read the last stages of this CTA's shared memory and
        // their commits to this CTA's barriers have landed
        for (int64_t q = g - STAGES < 0 ? 0 : g - STAGES; q < g; ++q)
            tc::mbar_wait(&empty[q % STAGES], (uint32_t)(q / STAGES) & 1u, deadline + 100000000ull);
    } else if (warp == 1 && lane == 0 && leader) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(PAIR_M, PAIR_N);
        int64_t g = 0;
        for (int j = 0;; ++j) {
            const int r = j % RING;
            const bool got = tc::mbar_wait(&sfull[r], (uint32_t)(j / RING) & 1u, deadline + 50000000ull);
            const int unit = got ? ring[r] : -1;
            tc::mbar_arrive(&sempty[r]);
            if (!got) *fail = 1;
            if (unit < 0) break;
            int tile, k0, k1, part, fix;
            unit_of<SPLIT>(unit, sp, KT, tile, k0, k1, part, fix);
            const int a = j % ACC;  // accumulator of this unit
            if (j >= ACC && !tc::mbar_wait_cluster(&tempty[a], (uint32_t)((j / ACC) - 1) & 1u, deadline)) {
                *fail = 1;
                tc::mma_commit_pair(&tfull[a], kBoth);
                continue;  // read the ring on to its end marker
            }
            tc::fence_after();
            const uint32_t acc_cols = tmem + (uint32_t)(a * PAIR_N);
            for (int kt = k0; kt < k1; ++kt, ++g) {
                const int s = (int)(g % STAGES);
                if (!tc::mbar_wait(&full[s], (uint32_t)(g / STAGES) & 1u, deadline)) {
                    *fail = 1;
                    break;
                }
                tc::fence_after();
                const uint32_t sa = tc::smem_u32(base + s * Cf::STAGE);
                const uint64_t adesc = tc::desc_sw128(sa);
                const uint64_t bdesc = tc::desc_sw128(sa + Cf::A_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    tc::mma_bf16_pair(acc_cols, adesc + 2ull * kk, bdesc + 2ull * kk, idesc,
                                      (uint32_t)((kt != k0) | (kk != 0)));
                tc::mma_commit_pair(&empty[s], kBoth);
            }
            tc::mma_commit_pair(&tfull[a], kBoth);  // also on failure, so both epilogues' waits complete
        }
    } else if (warp >= 2) {
        const int q = warp & 3;  // TMEM lane quadrant this warp may access
        for (int j = 0;; ++j) {
            const int r = j % RING;
            const bool got = tc::mbar_wait_cluster(&sfull[r], (uint32_t)(j / RING) & 1u, deadline + 50000000ull);
            const int unit = got ? ring[r] : -1;
            __syncwarp();
            if (lane == 0) tc::mbar_arrive_remote(tc::mapa(&sempty[r], 0));
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) *fail = 1;
                break;
            }
            if (unit < 0) break;
            const int a = j % ACC;
            const bool ok = tc::mbar_wait(&tfull[a], (uint32_t)(j / ACC) & 1u, deadline + 100000000ull);
            tc::fence_after();
            if (!__all_sync(0xffffffffu, ok && !*fail)) {
                if (lane == 0) *fail = 1;
                break;
            }
            int tile, k0, k1, part, fix;
            unit_of<SPLIT>(unit, sp, KT, tile, k0, k1, part, fix);
            const uint32_t trow = tmem + (uint32_t)(a * PAIR_N) + ((uint32_t)(q * 32) << 16);
            int tmi, tni;
            tile_coords(tile, tiles_m, tiles_n, group_m, tmi, tni);
            const int m0 = tmi * PAIR_M + (int)rank * HALF, n0 = tni * PAIR_N;
            // slot rows of a part: the CTA's 128 rows at rank x 128 of the 256-row slot
            const size_t slot_row = (size_t)rank * HALF + (size_t)(q * 32);
            float *crow = (!SPLIT || fix < 0)
                              ? C + (size_t)(m0 + q * 32 + lane) * (size_t)N + n0
                              : sp.ws + ((size_t)(fix * sp.parts + part) * PAIR_M + slot_row + lane) * PAIR_N;
            uint32_t ra[16], rb[16];
            tc::tmem_ld16(trow, ra);
            tc::tmem_ld_wait();
#pragma unroll
            for (int c = 0; c < CHUNKS; c += 2) {
                tc::tmem_ld16(trow + (uint32_t)((c + 1) * 16), rb);
                store_row16(crow + c * 16, ra);
                tc::tmem_ld_wait();
                if (c + 2 < CHUNKS) {
                    tc::tmem_ld16(trow + (uint32_t)((c + 2) * 16), ra);
                    store_row16(crow + (c + 1) * 16, rb);
                    tc::tmem_ld_wait();
                } else {
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive_remote(tc::mapa(&tempty[a], 0));  // this half is drained
                    store_row16(crow + (c + 1) * 16, rb);
                }
            }
            if (SPLIT && fix >= 0)
                split_arrive_reduce<PAIR_N>(sp, &sp.cnt[(fix * 2 + (int)rank) * EPI_WARPS + q],
                                            sp.ws + ((size_t)fix * sp.parts * PAIR_M + slot_row) * PAIR_N,
                                            (size_t)PAIR_M * PAIR_N, C + (size_t)(m0 + q * 32) * (size_t)N + n0, N,
                                            lane);
            if (warp == 2 && lane == 0) g_stamp(tm, false);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::cluster_sync();  // every remote arrival and every MMA into this CTA's TMEM is done
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc_pair(tmem, ACC * PAIR_N);
    }
    if (threadIdx.x == 0 && *fail) tm->status = IFR_ERR_TIMEOUT;
    g_exit(tm);
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&tm->tile_done, 1u) == gridDim.x - 1u) {
            atomicExch(&tm->tile_next, 0u);
            atomicExch(&tm->tile_done, 0u);
        }
    }
}

// ------------------------------------------------------------------ multicast pairs
// Variant 4: a cluster of two CTAs on two SMs takes two vertically adjacent 128 x 256
// tiles, (2p, n) and (2p + 1, n), which need the same 256 rows of B.  Each CTA
// loads its own 128 rows of A and one half (128 rows) of B, the half multicast into
// both CTAs' shared memory: 32 KiB of operands per SM per 64-wide K slice where a
// lone CTA needs 48 KiB.  Each CTA then issues its own cta_group::1 MMAs (M = 128,
// N = 256) into one of two 256-column accumulators and drains it with its own
// epilogue, as variant 3 does.
//   stage barriers  full[s]: one arrival (the CTA's own expect_tx of 48 KiB: its A,
//                   its B half and the other CTA's); a B half may land before the
//                   expect_tx of its phase (the pending arrival keeps the phase open);
//                   empty[s]: two arrivals, both CTAs' MMA commits (multicast), since
//                   a CTA's next copy into stage s also writes the other CTA's stage s
//   scheduling      the leader claims units (tile pairs) and writes each into both
//                   CTAs' rings, as the CTA-pair kernel does; the ring's release needs
//                   both MMA threads, both CTAs' epilogue warps and the other producer
// Bounded waits throughout; a final cluster barrier keeps each CTA resident until the
// other has finished writing into its shared memory.
template <int STAGES>
struct McCfg {
    static constexpr int A_BYTES = BM * BK * 2;        // 16 KiB
    static constexpr int B_BYTES = 256 * BK * 2;       // 32 KiB (both halves)
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
};

template <int STAGES>
__global__ void __launch_bounds__(GEMM_THREADS, 1) gemm_bf16_mc_kernel(const __grid_constant__ CUtensorMap ta,
                                                                       const __grid_constant__ CUtensorMap tb,
                                                                       float *__restrict__ C, int M, int N, int K,
                                                                       int group_m, DevTiming *tm) {
    using Cf = McCfg<STAGES>;
    constexpr int BN = 256, ACC = 2, CHUNKS = BN / 16;
    constexpr uint16_t kBoth = 3;
    extern __shared__ uint8_t g_smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)g_smem_raw + 1023u) & ~(uintptr_t)1023u);
    uint64_t *full = (uint64_t *)(base + STAGES * Cf::STAGE);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;   // [ACC]
    uint64_t *tempty = tfull + ACC;     // [ACC]
    uint64_t *sfull = tempty + ACC;     // [RING], both CTAs
    uint64_t *sempty = sfull + RING;    // [RING], leader
    int32_t *ring = (int32_t *)(sempty + RING);
    uint32_t *tmem_slot = (uint32_t *)(ring + RING);
    volatile int *fail = (volatile int *)(tmem_slot + 1);

    if (tc::cluster_nctarank() != 2) {
        if (threadIdx.x == 0) tm->status = IFR_ERR_LAUNCH;
        return;
    }
    const uint32_t rank = tc::cluster_ctarank();
    const bool leader = rank == 0;
    if (threadIdx.x == 0) g_stamp(tm, true);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = M / BM, tiles_n = N / BN, n_units = (tiles_m / 2) * tiles_n;
    const int KT = K / BK;
    const uint64_t deadline = ifr_gtimer() + kGemmTimeoutNs;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 2);
        }
        for (int a = 0; a < ACC; ++a) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], EPI_WARPS);
        }
        for (int r = 0; r < RING; ++r) {
            tc::mbar_init(&sfull[r], 1);
            tc::mbar_init(&sempty[r], 2 + 1 + 2 * EPI_WARPS);  // two MMA threads, the other producer, 8 epilogue warps
        }
        *fail = 0;
        tc::fence_mbar_init();
        tc::prefetch_tmap(&ta);
        tc::prefetch_tmap(&tb);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, ACC * BN);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    tc::cluster_sync();  // both CTAs' barriers are initialised before any remote arrival or multicast
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        int64_t g = 0;
        uint32_t next = blockIdx.x >> 1;  // leader: first unit = cluster index, later ones from the counter
        for (int j = 0;; ++j) {
            const int r = j % RING;
            int unit;
            if (leader) {
                if (j >= RING && !tc::mbar_wait_cluster(&sempty[r], (uint32_t)((j / RING) - 1) & 1u, deadline))
                    *fail = 1;
                unit = (*fail || next >= (uint32_t)n_units) ? -1 : (int)next;
                ring[r] = unit;
                tc::st_remote_s32(tc::mapa(&ring[r], 1), unit);
                tc::mbar_arrive(&sfull[r]);
                tc::mbar_arrive_remote(tc::mapa(&sfull[r], 1));
            } else {
                const bool got = tc::mbar_wait_cluster(&sfull[r], (uint32_t)(j / RING) & 1u, deadline + 50000000ull);
                unit = got ? ring[r] : -1;
                if (!got) *fail = 1;
                tc::mbar_arrive_remote(tc::mapa(&sempty[r], 0));
            }
            if (unit < 0) break;
            int pm, tni;
            tile_coords(unit, tiles_m / 2, tiles_n, group_m, pm, tni);
            const int m0 = (2 * pm + (int)rank) * BM, n0 = tni * BN;
            for (int kt = 0; kt < KT; ++kt, ++g) {
                const int s = (int)(g % STAGES);
                if (leader && kt == KT - 1) next = (gridDim.x >> 1) + atomicAdd(&tm->tile_next, 1u);
                // both CTAs' MMAs must have finished with stage s: this copy writes both
                if (g >= STAGES && !tc::mbar_wait_cluster(&empty[s], (uint32_t)((g / STAGES) - 1) & 1u, deadline)) {
                    *fail = 1;
                    break;
                }
                uint8_t *sa = base + s * Cf::STAGE;
                tc::mbar_arrive_expect_tx(&full[s], (uint32_t)Cf::STAGE);
                tc::tma_load_2d(sa, &ta, &full[s], kt * BK, m0);
                tc::tma_load_2d_mc(sa + Cf::A_BYTES + rank * (Cf::B_BYTES / 2), &tb, &full[s], kt * BK,
                                   n0 + (int)rank * (BN / 2), kBoth);
            }
        }
        // this CTA's own stages have landed (the other CTA's copies into it are covered
        // by the final cluster barrier, after its MMAs waited for them)
        for (int64_t q = g - STAGES < 0 ? 0 : g - STAGES; q < g; ++q)
            tc::mbar_wait(&full[q % STAGES], (uint32_t)(q / STAGES) & 1u, deadline + 100000000ull);
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
        int64_t g = 0;
        for (int j = 0;; ++j) {
            const int r = j % RING;
            const bool got = tc::mbar_wait_cluster(&sfull[r], (uint32_t)(j / RING) & 1u, deadline + 50000000ull);
            const int unit = got ? ring[r] : -1;
            tc::mbar_arrive_remote(tc::mapa(&sempty[r], 0));
            if (!got) *fail = 1;
            if (unit < 0) break;
            const int a = j % ACC;
            if (j >= ACC && !tc::mbar_wait(&tempty[a], (uint32_t)((j / ACC) - 1) & 1u, deadline)) {
                *fail = 1;
                tc::mma_commit(&tfull[a]);
                continue;
            }
            tc::fence_after();
            const uint32_t acc_cols = tmem + (uint32_t)(a * BN);
            for (int kt = 0; kt < KT; ++kt, ++g) {
                const int s = (int)(g % STAGES);
                if (!tc::mbar_wait(&full[s], (uint32_t)(g / STAGES) & 1u, deadline)) {
                    *fail = 1;
                    break;
                }
                tc::fence_after();
                const uint32_t sa = tc::smem_u32(base + s * Cf::STAGE);
                const uint64_t adesc = tc::desc_sw128(sa);
                const uint64_t bdesc = tc::desc_sw128(sa + Cf::A_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    tc::mma_bf16(acc_cols, adesc + 2ull * kk, bdesc + 2ull * kk, idesc, (uint32_t)((kt | kk) != 0));
                tc::mma_commit_mc(&empty[s], kBoth);
            }
            tc::mma_commit(&tfull[a]);
        }
    } else if (warp >= 2) {
        const int q = warp & 3;
        for (int j = 0;; ++j) {
            const int r = j % RING;
            const bool got = tc::mbar_wait_cluster(&sfull[r], (uint32_t)(j / RING) & 1u, deadline + 50000000ull);
            const int unit = got ? ring[r] : -1;
            __syncwarp();
            if (lane == 0) tc::mbar_arrive_remote(tc::mapa(&sempty[r], 0));
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) *fail = 1;
                break;
            }
            if (unit < 0) break;
            const int a = j % ACC;
            const bool ok = tc::mbar_wait(&tfull[a], (uint32_t)(j / ACC) & 1u, deadline + 100000000ull);
            tc::fence_after();
            if (!__all_sync(0xffffffffu, ok && !*fail)) {
                if (lane == 0) *fail = 1;
                break;
            }
            int pm, tni;
            tile_coords(unit, tiles_m / 2, tiles_n, group_m, pm, tni);
            const int m0 = (2 * pm + (int)rank) * BM, n0 = tni * BN;
            const uint32_t trow = tmem + (uint32_t)(a * BN) + ((uint32_t)(q * 32) << 16);
            float *crow = C + (size_t)(m0 + q * 32 + lane) * (size_t)N + n0;
            uint32_t ra[16], rb[16];
            tc::tmem_ld16(trow, ra);
            tc::tmem_ld_wait();
#pragma unroll
            for (int c = 0; c < CHUNKS; c += 2) {
                tc::tmem_ld16(trow + (uint32_t)((c + 1) * 16), rb);
                store_row16(crow + c * 16, ra);
                tc::tmem_ld_wait();
                if (c + 2 < CHUNKS) {
                    tc::tmem_ld16(trow + (uint32_t)((c + 2) * 16), ra);
                    store_row16(crow + (c + 1) * 16, rb);
                    tc::tmem_ld_wait();
                } else {
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&tempty[a]);
                    store_row16(crow + (c + 1) * 16, rb);
                }
            }
            if (warp == 2 && lane == 0) g_stamp(tm, false);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::cluster_sync();  // every multicast and remote arrival into this CTA has landed
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, ACC * BN);
    }
    if (threadIdx.x == 0 && *fail) tm->status = IFR_ERR_TIMEOUT;
    g_exit(tm);
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&tm->tile_done, 1u) == gridDim.x - 1u) {
            atomicExch(&tm->tile_next, 0u);
            atomicExch(&tm->tile_done, 0u);
        }
    }
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

// Variant 3 (two accumulators) is the one compiled with the split last wave.
template <int BN, int ST, int ACC>
const void *gemm_fn() {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gemm_bf16_kernel<BN, ST, ACC, ACC == 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             GemmCfg<BN, ST>::SMEM);
        attr = true;
    }
    return (const void *)gemm_bf16_kernel<BN, ST, ACC, ACC == 2>;
}

// The split of a variant-3 launch over `ctas` persistent CTAs: the tiles left over
// after the full waves (R = tiles mod ctas) become `parts` K ranges each when that
// fills the last wave better: parts = min(4, ctas / R, K / 2048), at least 2.  Each
// part then runs at least 32 K slices, enough to repay its partial tile's store and
// the reduction (measured: 2- and 4-part splits of 8 or fewer slices each made K = 512
// and K = 1024 launches slower than no split).
constexpr int kMinSlicesPerPart = 32;
GemmSplit split_for(int tiles, int ctas, int KT) {
    GemmSplit sp;
    memset(&sp, 0, sizeof sp);
    sp.parts = 1;
    const int R = tiles % ctas;
    if (R == 0) return sp;
    int parts = ctas / R;
    if (parts > 4) parts = 4;
    if (parts > KT / kMinSlicesPerPart) parts = KT / kMinSlicesPerPart;
    if (parts < 2) return sp;
    sp.full = tiles - R;
    sp.parts = parts;
    return sp;
}

// Workspace and counters of a split launch, owned by the context; the counters are
// zeroed when allocated, when the split changes and after a failed launch.
// slot_floats: floats of one part's partial tile; counters: counters per split tile.
int ensure_split(ifr_ctx *ctx, GemmSplit &sp, int tiles, size_t slot_floats, int counters, cudaStream_t stream) {
    if (sp.parts <= 1) return IFR_OK;
    const int R = tiles - sp.full;
    const size_t ws = (size_t)R * sp.parts * slot_floats * sizeof(float);
    const size_t nc = (size_t)R * counters;
    if (ws > ctx->gemm_ws_bytes) {
        if (ctx->gemm_ws) cudaFree(ctx->gemm_ws);
        ctx->gemm_ws = nullptr;
        ctx->gemm_ws_bytes = 0;
        IFR_CUDA(cudaMalloc((void **)&ctx->gemm_ws, ws));
        ctx->gemm_ws_bytes = ws;
    }
    if (nc > ctx->gemm_cnt_n) {
        if (ctx->gemm_cnt) cudaFree(ctx->gemm_cnt);
        ctx->gemm_cnt = nullptr;
        ctx->gemm_cnt_n = 0;
        IFR_CUDA(cudaMalloc((void **)&ctx->gemm_cnt, nc * sizeof(uint32_t)));
        ctx->gemm_cnt_n = nc;
        ctx->gemm_cnt_key = -1;
    }
    const int64_t key = (int64_t)R * 8 + sp.parts;
    if (key != ctx->gemm_cnt_key) {
        IFR_CUDA(cudaMemsetAsync(ctx->gemm_cnt, 0, ctx->gemm_cnt_n * sizeof(uint32_t), stream));
        ctx->gemm_cnt_key = key;
    }
    sp.ws = ctx->gemm_ws;
    sp.cnt = ctx->gemm_cnt;
    return IFR_OK;
}

template <int BN, int ST, int ACC>
int launch_gemm(ifr_ctx *ctx, const ifr_victim_cfg *c, cudaStream_t stream, int group_m, bool split, DevTiming *tm) {
    gemm_fn<BN, ST, ACC>();
    CUtensorMap ta, tb;
    int rc = make_map(&ta, c->in0, c->m, c->k, BM);
    if (rc) return rc;
    rc = make_map(&tb, c->in1, c->n, c->k, BN);
    if (rc) return rc;
    ifr_carveout(gemm_fn<BN, ST, ACC>());
    const int tiles = (int)((c->n / BN) * (c->m / BM));
    GemmSplit sp;
    memset(&sp, 0, sizeof sp);
    sp.parts = 1;
    if (split) {
        sp = split_for(tiles, g_num_sms, (int)(c->k / BK));
        rc = ensure_split(ctx, sp, tiles, (size_t)BM * BN, EPI_WARPS, stream);
        if (rc) return rc;
    }
    const int units = sp.parts > 1 ? sp.full + (tiles - sp.full) * sp.parts : tiles;
    const int grid = units < g_num_sms ? units : g_num_sms;
    gemm_bf16_kernel<BN, ST, ACC, ACC == 2><<<grid, GEMM_THREADS, GemmCfg<BN, ST>::SMEM, stream>>>(
        ta, tb, (float *)c->out, (int)c->m, (int)c->n, (int)c->k, group_m, sp, tm);
    return IFR_OK;
}

template <int ST, int ACC, bool SPLIT>
const void *gemm_pair_fn() {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gemm_bf16_pair_kernel<ST, ACC, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PairCfg<ST>::SMEM);
        attr = true;
    }
    return (const void *)gemm_bf16_pair_kernel<ST, ACC, SPLIT>;
}

template <int ST>
void pair_launch_cfg(cudaLaunchConfig_t *cfg, cudaLaunchAttribute *at, int grid, cudaStream_t stream) {
    memset(cfg, 0, sizeof(*cfg));
    memset(at, 0, sizeof(*at));
    cfg->gridDim = dim3((unsigned)grid);
    cfg->blockDim = dim3(GEMM_THREADS);
    cfg->dynamicSmemBytes = PairCfg<ST>::SMEM;
    cfg->stream = stream;
    at->id = cudaLaunchAttributeClusterDimension;
    at->val.clusterDim.x = 2;
    at->val.clusterDim.y = 1;
    at->val.clusterDim.z = 1;
    cfg->attrs = at;
    cfg->numAttrs = 1;
}

// CTA pairs the device can hold at once (pairs must sit in one GPC), asked once.
template <int ST, int ACC, bool SPLIT>
int pair_clusters() {
    static int n = 0;
    if (n == 0) {
        ifr_carveout(gemm_pair_fn<ST, ACC, SPLIT>());
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute at;
        pair_launch_cfg<ST>(&cfg, &at, 2 * (g_num_sms / 2), nullptr);
        int c = 0;
        if (cudaOccupancyMaxActiveClusters(&c, gemm_bf16_pair_kernel<ST, ACC, SPLIT>, &cfg) != cudaSuccess || c <= 0) {
            cudaGetLastError();
            c = g_num_sms / 2;
        }
        n = c < g_num_sms / 2 ? c : g_num_sms / 2;
    }
    return n;
}

// Split of a pair launch (SPLIT only) and its grid: one pair per unit, at most as
// many pairs as the device holds.
template <int ST, int ACC, bool SPLIT>
GemmSplit pair_split(const ifr_victim_cfg *c) {
    const int tiles = (int)((c->n / PAIR_N) * (c->m / PAIR_M));
    GemmSplit sp;
    memset(&sp, 0, sizeof sp);
    sp.parts = 1;
    if (SPLIT) sp = split_for(tiles, pair_clusters<ST, ACC, SPLIT>(), (int)(c->k / BK));
    return sp;
}

template <int ST, int ACC, bool SPLIT>
int pair_grid(const ifr_victim_cfg *c) {
    const int tiles = (int)((c->n / PAIR_N) * (c->m / PAIR_M));
    const GemmSplit sp = pair_split<ST, ACC, SPLIT>(c);
    const int units = sp.parts > 1 ? sp.full + (tiles - sp.full) * sp.parts : tiles;
    const int cl = pair_clusters<ST, ACC, SPLIT>();
    return 2 * (units < cl ? units : cl);
}

template <int ST, int ACC, bool SPLIT>
int launch_gemm_pair(ifr_ctx *ctx, const ifr_victim_cfg *c, cudaStream_t stream, int group_m, DevTiming *tm) {
    gemm_pair_fn<ST, ACC, SPLIT>();
    CUtensorMap ta, tb;
    int rc = make_map(&ta, c->in0, c->m, c->k, HALF);
    if (rc) return rc;
    rc = make_map(&tb, c->in1, c->n, c->k, HALF);
    if (rc) return rc;
    ifr_carveout(gemm_pair_fn<ST, ACC, SPLIT>());
    const int tiles = (int)((c->n / PAIR_N) * (c->m / PAIR_M));
    GemmSplit sp = pair_split<ST, ACC, SPLIT>(c);
    rc = ensure_split(ctx, sp, tiles, (size_t)PAIR_M * PAIR_N, 2 * EPI_WARPS, stream);
    if (rc) return rc;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at;
    pair_launch_cfg<ST>(&cfg, &at, pair_grid<ST, ACC, SPLIT>(c), stream);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, gemm_bf16_pair_kernel<ST, ACC, SPLIT>, ta, tb, (float *)c->out,
                                             (int)c->m, (int)c->n, (int)c->k, group_m, sp, tm);
    return e == cudaSuccess ? IFR_OK : IFR_ERR_LAUNCH;
}

template <int ST>
const void *gemm_mc_fn() {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gemm_bf16_mc_kernel<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, McCfg<ST>::SMEM);
        attr = true;
    }
    return (const void *)gemm_bf16_mc_kernel<ST>;
}

template <int ST>
void mc_launch_cfg(cudaLaunchConfig_t *cfg, cudaLaunchAttribute *at, int grid, cudaStream_t stream) {
    memset(cfg, 0, sizeof(*cfg));
    memset(at, 0, sizeof(*at));
    cfg->gridDim = dim3((unsigned)grid);
    cfg->blockDim = dim3(GEMM_THREADS);
    cfg->dynamicSmemBytes = McCfg<ST>::SMEM;
    cfg->stream = stream;
    at->id = cudaLaunchAttributeClusterDimension;
    at->val.clusterDim.x = 2;
    at->val.clusterDim.y = 1;
    at->val.clusterDim.z = 1;
    cfg->attrs = at;
    cfg->numAttrs = 1;
}

// Clusters of the multicast kernel the device holds at once, asked once.
template <int ST>
int mc_clusters() {
    static int n = 0;
    if (n == 0) {
        ifr_carveout(gemm_mc_fn<ST>());
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute at;
        mc_launch_cfg<ST>(&cfg, &at, 2 * (g_num_sms / 2), nullptr);
        int c = 0;
        if (cudaOccupancyMaxActiveClusters(&c, gemm_bf16_mc_kernel<ST>, &cfg) != cudaSuccess || c <= 0) {
            cudaGetLastError();
            c = g_num_sms / 2;
        }
        n = c < g_num_sms / 2 ? c : g_num_sms / 2;
    }
    return n;
}

template <int ST>
int mc_grid(const ifr_victim_cfg *c) {
    const int units = (int)((c->m / 256) * (c->n / 256));
    const int cl = mc_clusters<ST>();
    return 2 * (units < cl ? units : cl);
}

template <int ST>
int launch_gemm_mc(const ifr_victim_cfg *c, cudaStream_t stream, int group_m, DevTiming *tm) {
    gemm_mc_fn<ST>();
    CUtensorMap ta, tb;
    int rc = make_map(&ta, c->in0, c->m, c->k, BM);
    if (rc) return rc;
    rc = make_map(&tb, c->in1, c->n, c->k, 128);  // one half of a 256-row B panel per copy
    if (rc) return rc;
    ifr_carveout(gemm_mc_fn<ST>());
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at;
    mc_launch_cfg<ST>(&cfg, &at, mc_grid<ST>(c), stream);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, gemm_bf16_mc_kernel<ST>, ta, tb, (float *)c->out, (int)c->m,
                                             (int)c->n, (int)c->k, group_m, tm);
    return e == cudaSuccess ? IFR_OK : IFR_ERR_LAUNCH;
}

template <int BN>
const void *gemm_group_fn() {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gemm_bf16_group_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             GemmCfg<BN, 3>::SMEM);
        attr = true;
    }
    return (const void *)gemm_bf16_group_kernel<BN>;
}

}  // namespace

int ifr_gemm_shape(const ifr_victim_cfg *c, VictimShape *s) {
    if (g_num_sms == 0) cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, 0);
    s->flops = 2.0 * (double)c->m * (double)c->n * (double)c->k;
    s->bytes = 2.0 * ((double)c->m + (double)c->n) * (double)c->k + 4.0 * (double)c->m * (double)c->n;
    s->uses_tensor = 1;
    s->block = GEMM_THREADS;
    if (c->variant == 2) {
        s->fn = gemm_pair_fn<6, 2, true>();
        s->grid = pair_grid<6, 2, true>(c);
        s->smem = PairCfg<6>::SMEM;
        s->tmem_cols = 2 * PAIR_N;
        return IFR_OK;
    }
    if (c->variant == 4) {
        s->fn = gemm_mc_fn<4>();
        s->grid = mc_grid<4>(c);
        s->smem = McCfg<4>::SMEM;
        s->tmem_cols = 512;
        return IFR_OK;
    }
    const bool wide = c->n % 256 == 0;
    const int BN = wide ? 256 : 128;
    const int tiles = (int)((c->n / BN) * (c->m / BM));
    if (c->variant == 3) {
        s->fn = wide ? gemm_fn<256, 4, 2>() : gemm_fn<128, 4, 2>();
        const GemmSplit sp = split_for(tiles, g_num_sms, (int)(c->k / BK));
        const int units = sp.parts > 1 ? sp.full + (tiles - sp.full) * sp.parts : tiles;
        s->grid = units < g_num_sms ? units : g_num_sms;
        s->smem = wide ? GemmCfg<256, 4>::SMEM : GemmCfg<128, 4>::SMEM;
        s->tmem_cols = 2 * BN;
        return IFR_OK;
    }
    const bool deep = c->variant == 1;
    s->fn = wide ? (deep ? gemm_fn<256, 4, 1>() : gemm_fn<256, 3, 1>())
                 : (deep ? gemm_fn<128, 4, 1>() : gemm_fn<128, 3, 1>());
    s->grid = tiles < g_num_sms ? tiles : g_num_sms;
    s->smem = wide ? (deep ? GemmCfg<256, 4>::SMEM : GemmCfg<256, 3>::SMEM)
                   : (deep ? GemmCfg<128, 4>::SMEM : GemmCfg<128, 3>::SMEM);
    s->tmem_cols = BN;
    return IFR_OK;
}

int ifr_gemm_enqueue(ifr_ctx *ctx, const ifr_victim_cfg *c, cudaStream_t stream, DevTiming *tm) {
    g_num_sms = ctx->info.num_sms;
    if (c->m > 65535 * BM || c->n > (1ll << 30) || c->k > (1ll << 30)) return IFR_ERR_ARG;
    const double operand_bytes = 2.0 * ((double)c->m + (double)c->n) * (double)c->k;
    const int gm = operand_bytes > (double)ctx->info.l2_bytes ? GROUP_M : 1;
    if (c->variant == 2) return launch_gemm_pair<6, 2, true>(ctx, c, stream, gm, tm);
    if (c->variant == 4) return launch_gemm_mc<4>(c, stream, gm, tm);
    const bool wide = c->n % 256 == 0;
    if (c->variant == 3)
        return wide ? launch_gemm<256, 4, 2>(ctx, c, stream, gm, true, tm)
                    : launch_gemm<128, 4, 2>(ctx, c, stream, gm, true, tm);
    const bool deep = c->variant == 1;
    if (wide)
        return deep ? launch_gemm<256, 4, 1>(ctx, c, stream, gm, false, tm)
                    : launch_gemm<256, 3, 1>(ctx, c, stream, gm, false, tm);
    return deep ? launch_gemm<128, 4, 1>(ctx, c, stream, gm, false, tm)
                : launch_gemm<128, 3, 1>(ctx, c, stream, gm, false, tm);
}

// Grouping key of a GEMM victim (0 = alone): variant-0 GEMMs group by tile width.
int ifr_gemm_group_key(const ifr_victim_cfg *c) {
    if (c->variant != 0 || c->grid) return 0;
    return c->n % 256 == 0 ? 402 : 401;
}

// K grouped launches of GEMM victims vs[0..n-1] of one tile width (validated by the
// caller), victim i stamping into tms[i].
int ifr_gemm_enqueue_group(ifr_ctx *ctx, const ifr_victim_cfg *const *vs, DevTiming *const *tms, int n,
                           cudaStream_t stream) {
    if (n <= 0 || n > IFR_GROUP_MAX) return IFR_ERR_ARG;
    g_num_sms = ctx->info.num_sms;
    const int key = ifr_gemm_group_key(vs[0]);
    if (key <= 0) return IFR_ERR_ARG;
    const bool wide = key == 402;
    const int BN = wide ? 256 : 128;
    GemmGroup g;
    memset(&g, 0, sizeof g);
    int64_t tile0 = 0;
    for (int i = 0; i < n; ++i) {
        const ifr_victim_cfg *c = vs[i];
        if (ifr_gemm_group_key(c) != key || c->m > 65535 * BM || c->n > (1ll << 30) || c->k > (1ll << 30))
            return IFR_ERR_ARG;
        GemmProblem &pb = g.p[i];
        int rc = make_map(&pb.ta, c->in0, c->m, c->k, BM);
        if (!rc) rc = make_map(&pb.tb, c->in1, c->n, c->k, BN);
        if (rc) return rc;
        pb.C = (float *)c->out;
        pb.tm = tms[i];
        pb.N = (int32_t)c->n;
        pb.K = (int32_t)c->k;
        pb.tiles_m = (int32_t)(c->m / BM);
        pb.tiles_n = (int32_t)(c->n / BN);
        pb.tile0 = (int32_t)tile0;
        const double operand_bytes = 2.0 * ((double)c->m + (double)c->n) * (double)c->k;
        pb.group_m = operand_bytes > (double)ctx->info.l2_bytes ? GROUP_M : 1;
        tile0 += (int64_t)pb.tiles_m * pb.tiles_n;
        if (tile0 >= (1ll << 31)) return IFR_ERR_ARG;
    }
    g.n = n;
    g.total = (int32_t)tile0;
    const void *fn = wide ? gemm_group_fn<256>() : gemm_group_fn<128>();
    ifr_carveout(fn);
    const int grid = g.total < g_num_sms ? g.total : g_num_sms;
    const int K = vs[0]->repeats > 0 ? vs[0]->repeats : 1;
    for (int rep = 0; rep < K; ++rep) {
        if (wide)
            gemm_bf16_group_kernel<256><<<grid, GEMM_THREADS, GemmCfg<256, 3>::SMEM, stream>>>(g);
        else
            gemm_bf16_group_kernel<128><<<grid, GEMM_THREADS, GemmCfg<128, 3>::SMEM, stream>>>(g);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return ifr_cuda_fail(e, "grouped GEMM launch", __FILE__, __LINE__);
        ctx->kernel_launches += 1;
    }
    return IFR_OK;
}

// After a launch that failed part-way the split counters may be off by a few
// arrivals: the next split launch starts from zero.
void ifr_gemm_forget_split(ifr_ctx *ctx) { ctx->gemm_cnt_key = -1; }

int ifr_preload_gemm() {
    const void *fns[] = {gemm_fn<128, 3, 1>(), gemm_fn<256, 3, 1>(), gemm_fn<128, 4, 1>(), gemm_fn<256, 4, 1>(),
                         gemm_fn<128, 4, 2>(), gemm_fn<256, 4, 2>(), gemm_pair_fn<6, 2, true>(), gemm_mc_fn<4>(),
                         gemm_group_fn<128>(), gemm_group_fn<256>()};
    for (const void *f : fns) {
        int rc = ifr_preload(f);
        if (rc) return rc;
    }
    return IFR_OK;
}
