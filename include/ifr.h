/*
 * ifr.h — C ABI of libifr, the B300 (sm_103a) interference-sensitivity library.
 *
 * The method (Elvinger, Strati, Enright Jerger, Klimovic, "Understanding GPU
 * Resource Interference One Level Deeper", SoCC '25):
 *   - Sec. 1 and Sec. 4.1: quantify a workload's sensitivity to each GPU resource
 *     by colocating it with custom stressor benchmarks, each of which stresses one
 *     resource and holds a constant interference level for the whole life of the
 *     colocated workload; intra-SM colocation uses CUDA streams, inter-SM
 *     colocation partitions the SMs.
 *   - Sec. 4.3 / 4.4: slowdown = latency colocated / latency in isolation.
 *   - Sec. 5.1: a kernel-level estimator that combines each kernel's metrics and
 *     resource sensitivity to predict its slowdown.
 *
 * Conventions for every entry point:
 *   - Return value: IFR_OK (0) or a negative IFR_ERR_* status; nothing aborts the
 *     process.  ifr_strerror() names a status.
 *   - Device pointers are plain CUDA device addresses owned by the caller (for
 *     example torch tensors' data_ptr()); the library never frees them.  Host
 *     pointers are plain host memory owned by the caller.
 *   - Streams are cudaStream_t values passed as void*; NULL selects the context's
 *     own stream for that role.
 *   - The context (ifr_ctx) owns its streams, per-run device scratch (flags,
 *     counters, per-block logs), events and green contexts.  One context per host
 *     thread; calls on one context are not thread-safe.
 *   - Every device-side wait in the library's kernels is bounded by a deadline
 *     (%globaltimer) and an iteration cap; on expiry the kernel records
 *     IFR_ERR_TIMEOUT / IFR_ERR_NOT_RESIDENT and returns.
 */
#ifndef IFR_H
#define IFR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IFR_ABI_VERSION 4

/* ---- status codes ------------------------------------------------------- */
#define IFR_OK 0
#define IFR_ERR_ARG (-1)          /* invalid argument (null, size, alignment, kind) */
#define IFR_ERR_CUDA (-2)         /* a CUDA runtime/driver call failed */
#define IFR_ERR_TIMEOUT (-3)      /* a device or host wait reached its deadline */
#define IFR_ERR_NOT_RESIDENT (-4) /* the stressor never became resident before the victim */
#define IFR_ERR_LAUNCH (-5)       /* a kernel launch was rejected */
#define IFR_ERR_BOUNDS (-6)       /* a checked build caught an out-of-range index */
#define IFR_ERR_UNSUPPORTED (-7)  /* feature unavailable on this device / driver */
#define IFR_ERR_NOMEM (-8)        /* context scratch allocation failed */
#define IFR_ERR_CAPACITY (-9)     /* output array too small / no free slot */
#define IFR_ERR_INVALID_CELL (-10) /* a measurement violated the constant-interference rule */
#define IFR_ERR_HOL (-11)         /* no victim block could become co-resident with the stressor
                                     (block-scheduler head-of-line blocking, Sec. 4.2); the
                                     stressor gave up so the victim could run */

#define IFR_MAX_STRESSORS 16
#define IFR_MAX_LEVELS 16
#define IFR_MAX_SMS 256

typedef struct ifr_ctx ifr_ctx;

/* ---- context ------------------------------------------------------------ */
typedef struct {
    int32_t device, num_sms, cc_major, cc_minor;
    int64_t l2_bytes;              /* cudaDevAttrL2CacheSize */
    int32_t smem_per_sm;           /* bytes */
    int32_t smem_per_block_optin;  /* bytes */
    int32_t regs_per_sm, max_threads_per_sm, max_blocks_per_sm;
    int32_t sm_clock_khz, mem_clock_khz, mem_bus_width_bits;
    int64_t global_mem_bytes;
    char name[128];
} ifr_device_info;

/* Create a context on CUDA device `device`: queries the device, creates the
 * stressor / victim / control streams and allocates per-slot scratch.  The
 * device must be sm_100-family (this build carries sm_103a code only).
 * Errors: IFR_ERR_ARG (null out), IFR_ERR_CUDA, IFR_ERR_UNSUPPORTED (wrong arch). */
int ifr_init(int device, ifr_ctx **out);
/* Destroy a context; waits (bounded) for its streams.  NULL is a no-op. */
void ifr_shutdown(ifr_ctx *ctx);
/* Static string for a status code. */
const char *ifr_strerror(int status);
int ifr_abi_version(void);
int ifr_device_query(ifr_ctx *ctx, ifr_device_info *out);
/* Number of kernels this context has enqueued so far (each replay of a captured
 * graph adds its kernel nodes).  Errors: IFR_ERR_ARG. */
int ifr_launch_count(ifr_ctx *ctx, uint64_t *out);

/* ---- stressors (Sec. 3, Sec. 4.2-4.4) ----------------------------------- */
/* The paper's stressors: block-scheduler (sleep) kernel Sec. 4.2; compute kernel
 * (independent fp32 multiplies, ILP knob) Sec. 3 and Sec. 4.4.2; copy kernel over
 * an L2-sized or HBM-sized buffer Sec. 4.3; n-strided shared-memory copy Sec.
 * 4.4.1.  The tensor-pipe stressor follows the pipe-utilisation metric of
 * Sec. 2.2.  Each kernel folds what it touched into a checksum (see the oracle). */
typedef enum {
    IFR_S_SCHED = 0,    /* short blocks: block dispatch and SM block slots */
    IFR_S_FMA = 1,      /* dependent fp32 FMA chains, ILP independent chains/thread */
    IFR_S_TENSOR = 2,   /* BF16 tcgen05 MMA loop, 128x128x64 tiles, TMEM accumulator */
    IFR_S_SMEM_CF = 3,  /* shared-memory ld/st, conflict-free (1 wavefront / request) */
    IFR_S_SMEM_32W = 4, /* shared-memory ld/st, 32-way bank conflicts */
    IFR_S_L2 = 5,       /* streaming XOR read of an L2-resident buffer */
    IFR_S_HBM = 6,      /* streaming XOR read of an HBM-sized buffer */
    IFR_S_FP64 = 7,     /* dependent fp64 multiply chains (Sec. 4.4.3), ILP chains/thread */
    IFR_S_SLEEP = 8,    /* blocks that hold their SM slot and sleep (Sec. 4.2 sleep kernel) */
    IFR_S_COUNT = 9
} ifr_stressor_kind;

typedef struct {
    int32_t kind;            /* ifr_stressor_kind */
    int32_t sm_count;        /* SMs the stressor may occupy: 0 = none (harness-only
                                launch, "intensity 0"), num_sms = all.  The SMs are
                                spread evenly over the SM id range. */
    int32_t blocks_per_sm;   /* persistent blocks per allowed SM (0 = kind default) */
    int32_t block;           /* threads per block (0 = kind default) */
    int32_t ilp;             /* FMA / FP64: independent chains per thread (1,2,4,8; 0 = 4) */
    int32_t smem_ways;       /* SMEM: bank-conflict degree 1..32 power of 2 (0 = kind) */
    float duty;              /* active fraction of each period, (0, 1]; 0 or 1 = always */
    int32_t period_ns;       /* duty-cycle period (0 = 100000); SLEEP: sleep per round */
    int64_t working_set_bytes; /* L2/HBM: bytes of buf streamed; multiple of block*64.
                                  SLEEP: dynamic shared memory held per block
                                  (<= the device's opt-in limit per block - 1 KiB) */
    const void *buf;         /* L2/HBM: device buffer of >= working_set_bytes, 16-B aligned */
    uint64_t seed;           /* private seed for FMA / SMEM / TENSOR / SCHED values */
    int64_t max_rounds;      /* > 0: each block stops after this many rounds (fixed work);
                                0: run until stopped or the deadline */
    int32_t sched_blocks;    /* SCHED: blocks per launch (0 = 100000) */
    int32_t sched_launches;  /* SCHED: launches enqueued (0 = 64) */
    int32_t sched_cycles;    /* SCHED: busy cycles per block (0 = 100) */
    int32_t mask_mode;       /* 0: sm_count SMs spread evenly over the SM ids (%smid filter);
                                1: any SM of the green-context partition that owns the launch
                                   stream (needs an active ifr_partition; sm_count = SMs to
                                   claim, at most the larger partition's count);
                                2: exactly the SMs set in sm_mask (%smid filter), e.g. two
                                   disjoint partitions as in Sec. 4.3's inter-SM runs;
                                   sm_count must equal the number of bits set */
    uint64_t deadline_ns;    /* device-side limit on the run (0 = 2 s) */
    uint32_t sm_mask[IFR_MAX_SMS / 32]; /* mask_mode 2: bit s of word s/32 allows SM id s */
    int32_t staging;         /* L2/HBM: 0 = loads into registers, no shared memory
                                (default): a thread loads the first word of each of its
                                16-byte groups, which brings every 32-byte sector of the
                                chunk into the SM; the checksum folds those words;
                                1 = TMA bulk copies (cp.async.bulk) of whole chunks into a ring
                                in shared memory of about 96 KiB per block (2 to 6 stages of
                                block x 64 bytes), folded from there (the checksum folds
                                quarter pass mod 4 of every chunk).  The ring keeps victim
                                blocks that need much shared memory off the stressor's SMs.
                                Other kinds: 0 */
    int32_t reserved;
} ifr_stressor_cfg;

typedef struct {
    uint32_t checksum;       /* XOR of the per-block checksums (SCHED: of all blocks) */
    int32_t status;          /* first error recorded by any block, or IFR_OK */
    uint64_t rounds;         /* rounds summed over active blocks (SCHED: working blocks) */
    uint64_t work;           /* kind units: chunks (L2/HBM), FMA / FP64 steps/thread-chain, rounds (SLEEP),
                                smem ld/st pairs/lane, tile MMAs, busy blocks (SCHED) */
    uint64_t t_start_ns;     /* earliest active-block start (%globaltimer) */
    uint64_t t_start_last_ns;/* latest active-block start */
    uint64_t t_end_first_ns; /* earliest active-block end */
    uint64_t t_end_ns;       /* latest active-block end */
    int32_t blocks_launched; /* grid size (SCHED: blocks over all launches) */
    int32_t blocks_active;   /* blocks that passed the SM filter and worked */
    int32_t sms_used;        /* distinct SMs with an active block */
    int32_t planned_active;  /* sm_count * blocks_per_sm (work-split stride) */
    double elapsed_ms;       /* cudaEvent time from launch to completion */
} ifr_stressor_result;
/* SCHED (a chain of short-block launches): one working block in 256 records its start
 * and end; t_start_ns = t_start_last_ns is the first recorded start, and t_end_ns =
 * t_end_first_ns is the later of the last recorded end and the first time one block
 * in 4096 saw the stop request (the chain was still running then). */

typedef struct {
    uint64_t t_start_ns, t_end_ns; /* %globaltimer at block entry / exit */
    uint64_t rounds;               /* rounds this block completed */
    uint64_t work;                 /* kind units this block completed */
    uint32_t checksum;             /* per-block checksum (FMA: after round 0) */
    uint32_t checksum2;            /* FMA: after the last round; else 0 */
    uint32_t smid;
    int32_t index;                 /* active-block index k (claim order) */
    int32_t status;
    uint32_t reserved;
} ifr_block_log;

/* Launch a stressor on `stream` (NULL = the context's stressor stream) and return
 * a handle.  Non-blocking.  Persistent kinds launch num_sms * blocks_per_sm
 * blocks; a block that lands on an SM outside the mask, or beyond blocks_per_sm
 * on its SM, exits at once.  Runs until ifr_stressor_stop, max_rounds, or the
 * deadline.  Errors: IFR_ERR_ARG, IFR_ERR_CAPACITY (no free slot), IFR_ERR_LAUNCH. */
int ifr_stressor_launch(ifr_ctx *ctx, const ifr_stressor_cfg *cfg, void *stream, int *handle_out);
/* Ask the stressor to stop.  stream != NULL: the stop is enqueued on that stream
 * (it takes effect after the work queued there, e.g. the victim launches);
 * stream == NULL: the stop is written at once from the host. */
int ifr_stressor_stop(ifr_ctx *ctx, int handle, void *stream);
/* Wait (host, bounded by timeout_ms; 0 = 10000) for the stressor to finish, then
 * fill *out.  On host timeout the stop flag is set and IFR_ERR_TIMEOUT returned. */
int ifr_stressor_wait(ifr_ctx *ctx, int handle, int timeout_ms, ifr_stressor_result *out);
/* Copy the per-block logs of a finished stressor (active blocks, index order). */
int ifr_stressor_block_logs(ifr_ctx *ctx, int handle, ifr_block_log *out, int cap, int *n_out);
/* Free the slot of a finished stressor. */
int ifr_stressor_release(ifr_ctx *ctx, int handle);

/* Allocation-free fixed-work run of the L2/HBM stream stressor (the paper has no
 * counterpart: this is a convenience of the library).  Some callers cannot call
 * cudaMalloc: latency-critical loops that must not block on the device allocator
 * (cudaMalloc can synchronise the device), and hosts that
 * own a fixed device-memory budget and so never create an ifr_ctx (ifr_init
 * allocates).  This entry point needs no context and allocates nothing: its
 * control state (stop flag, counters, per-SM claim table) is a 4 KiB file-scope
 * device array that every GPU loading the library keeps until the process exits.
 * Arguments: kind IFR_S_L2 or IFR_S_HBM; buf / working_set_bytes / block as in
 * ifr_stressor_cfg; sm_count SMs (spread as in ifr_stressor_cfg) with
 * blocks_per_sm blocks each; max_rounds > 0 rounds per block (fixed work, no stop
 * request exists); deadline_ns as in ifr_stressor_cfg (0 = 2 s); stream a
 * cudaStream_t (NULL = legacy default stream); logs_out a caller-owned device
 * array of logs_cap >= sm_count * blocks_per_sm records, written in active-index
 * order (unclaimed slots keep index -1).  Asynchronous: synchronise `stream`
 * before reading logs_out.  The first call on a device looks up the array's
 * device address with that device current and loads the entry point's kernels,
 * so make it before any stream capture.  `stream` must belong to the current
 * device.  The looked-up address is kept for the life of the process: calls after
 * a cudaDeviceReset of that device are not supported.
 * All calls share the array, which keeps the last call's contents (the call
 * clears it on the stream first): calls whose kernels overlap on the GPU race.
 * Errors: IFR_ERR_ARG (kind, pointer, alignment, size, rounds), IFR_ERR_CAPACITY
 * (logs_cap too small, or a device with more than IFR_MAX_SMS SMs), IFR_ERR_CUDA. */
int ifr_stream_stressor_noalloc(int kind, const void *buf, int64_t working_set_bytes, int sm_count,
                                int blocks_per_sm, int block, int64_t max_rounds, uint64_t deadline_ns,
                                void *stream, ifr_block_log *logs_out, int logs_cap);

/* ---- victims ------------------------------------------------------------ */
/* Workloads whose slowdown is measured (Sec. 4: the paper uses LLM decode and
 * torch.mm; this library uses kernels with textbook definitions). */
typedef enum {
    IFR_V_TRIAD = 0,     /* a[i] = b[i] + s*c[i]; fp32; n elements */
    IFR_V_GEMM = 1,      /* C[m][n] = sum_k A[m][k] B[n][k]; A MxK, B NxK bf16; C fp32 */
    IFR_V_GEMV = 2,      /* y[r] = sum_c A[r][c] x[c]; A m x k bf16 row-major; y fp32 */
    IFR_V_LAYERNORM = 3, /* per row (m rows, n cols): (x-mean)/sqrt(var+eps); fp32 */
    IFR_V_SOFTMAX = 4,   /* per row (m rows, n cols): exp(x-max)/sum; fp32 */
    IFR_V_HIST = 5,      /* 256-bin histogram of key & 255; n int32 keys; u32 bins */
    IFR_V_COUNT = 6
} ifr_victim_kind;

typedef struct {
    int32_t kind;          /* ifr_victim_kind */
    int32_t repeats;       /* K back-to-back launches per measurement (0 = 1) */
    int64_t m, n, k;       /* shapes, see ifr_victim_kind */
    float scalar;          /* TRIAD s */
    float eps;             /* LAYERNORM eps (0 = 1e-5) */
    const void *in0;       /* TRIAD b | GEMM A | GEMV A | LN/SOFTMAX x | HIST keys */
    const void *in1;       /* TRIAD c | GEMM B | GEMV x */
    void *out;             /* TRIAD a | GEMM C | GEMV y | LN/SOFTMAX y | HIST bins */
    int32_t grid;          /* blocks (0 = kind default) */
    int32_t block;         /* threads per block (0 = kind default) */
    int32_t variant;       /* GEMM: 0 = colocation-friendly (3 TMA stages, 145 KiB of shared
                              memory: leaves room for a stressor block, Sec. 5.3),
                              1 = throughput (4 stages, 193 KiB: more operand bytes in
                              flight, but no shared-memory stressor block fits beside it),
                              2 = CTA pairs, the fastest variant (a 2-CTA cluster per
                              256 x 256 tile with tcgen05 cta_group::2, 6 stages of 32
                              KiB per SM, 193 KiB; two 256-column accumulators per SM;
                              the split last wave of variant 3 over pair tiles, with K
                              ranges of at least 2048; m and n multiples of 256, else
                              IFR_ERR_ARG).  The pair's TMEM allocation needs the same
                              512 columns free on both SMs: beside other TMEM users (the
                              tensor stressor) it can wait until they exit, so it is for
                              solo use (ifr_victim_launch); ifr_sweep, ifr_corun and
                              ifr_colocate refuse it with IFR_ERR_ARG.
                              3 = throughput, two accumulators: variant 1 (4 stages) with
                              two 256-column TMEM accumulators, so the next tile's MMAs
                              overlap the epilogue, and, when the tiles leave the last wave
                              of CTAs part-empty, the left-over tiles split into 2-4 K
                              ranges of at least 2048 (partial tiles in a context-owned
                              workspace, reduced in a fixed order by the last range);
                              4 = multicast pairs: a 2-CTA cluster takes two vertically
                              adjacent 128 x 256 tiles and loads each half of their shared
                              256 rows of B once, multicast into both CTAs (m and n
                              multiples of 256, else IFR_ERR_ARG), two accumulators.
                              Variants 3 and 4 hold all 512 TMEM columns of an SM: solo
                              use only, refused like variant 2.
                              GEMV: 0 = one warp per row, 16-byte loads into registers;
                              1 = rows streamed into shared memory by bulk copies (each
                              warp a ring of two 4 KiB segments; x in shared memory too,
                              80 KiB per block at k = 8192), for solo use: ifr_sweep,
                              ifr_corun and ifr_colocate refuse it with IFR_ERR_ARG.
                              Other kinds: 0. */
    int32_t reserved;
} ifr_victim_cfg;

typedef struct {
    uint64_t t_start_ns;   /* earliest block entry over the K launches (%globaltimer) */
    uint64_t t_end_ns;     /* latest block exit over the K launches */
    double event_ms;       /* cudaEvent time around the K launches */
    int32_t status;        /* IFR_OK, or IFR_ERR_NOT_RESIDENT from the residency wait */
    int32_t sms_touched;   /* distinct SMs that ran a victim block */
    int32_t blocks;        /* blocks executed over the K launches */
    int32_t repeats;       /* K */
} ifr_timing;

/* Run K back-to-back launches of a victim on `stream` (NULL = context victim
 * stream), wait for them and fill *out (may be NULL to skip timing read-back,
 * then the call still synchronises).  Errors: IFR_ERR_ARG (shape, null or
 * misaligned pointer), IFR_ERR_LAUNCH, IFR_ERR_CUDA. */
int ifr_victim_launch(ifr_ctx *ctx, const ifr_victim_cfg *cfg, void *stream, ifr_timing *out);

/* ---- SM partitions (green contexts; Sec. 4.1 inter-SM colocation) ------ */
/* The paper colocates across SMs with CUDA green contexts, each a disjoint SM set
 * with its own stream (Sec. 4.1, 4.3).  ifr_partition splits the device's SMs into
 * two such partitions: one of at least `victim_sms` SMs (rounded up to the split
 * granularity) and one of the rest.  While the split is active the context's
 * victim stream belongs to the first and its stressor stream to the second, so
 * every sweep, ifr_colocate and ifr_stressor_pair run places victims and stressors
 * (or pair A on the stressor side, pair B on the victim side) on disjoint SMs;
 * stressors then use mask_mode 1.  flags: 1 = split each SM on its own (finer
 * granularity, no SM co-scheduling guarantees), 0 = the driver's default split.
 * Errors: IFR_ERR_ARG (victim_sms out of range, a split already active),
 * IFR_ERR_UNSUPPORTED (no green-context support), IFR_ERR_CUDA. */
typedef struct {
    int32_t victim_sms;    /* SMs of the victim partition */
    int32_t stressor_sms;  /* SMs of the stressor partition */
} ifr_partition_info;
int ifr_partition(ifr_ctx *ctx, int victim_sms, int flags, ifr_partition_info *out);
/* Undo ifr_partition (after synchronising the device); no-op without a split. */
int ifr_partition_release(ifr_ctx *ctx);

/* ---- two stressors against each other (Sec. 3 pitfalls, Sec. 4.3, Sec. 4.4.3) -- */
/* The paper's kernel-against-kernel experiments colocate two fixed-work kernels
 * and compare each one's latency with its latency alone: two compute kernels at
 * 6.25 % achieved occupancy (Pitfall 1), a compute kernel beside a copy kernel
 * (Pitfall 2), two copy kernels on disjoint SM partitions over growing data
 * (L2 pollution, Sec. 4.3), and two fp64 compute kernels whose speedup
 * sequential/colocated tracks the summed pipe utilisation (Table 3).
 * ifr_stressor_pair runs A alone, B alone, then A and B released at the same
 * instant on two streams (both streams wait on one event recorded after a short
 * device-side gate, so neither starts first by a host launch latency).  A runs on
 * the context's stressor stream and B on its victim stream, alone and together, so
 * under ifr_partition each stays in its own partition.  Both
 * configurations must be fixed-work (max_rounds > 0) persistent kinds (not
 * IFR_S_SCHED); their SM sets (mask_mode 0 or 2) may overlap or be disjoint.
 * Spans are %globaltimer first-block start to last-block end. */
typedef struct {
    ifr_stressor_result solo_a, solo_b;  /* each alone */
    ifr_stressor_result co_a, co_b;      /* released together */
    double solo_a_ns, solo_b_ns;         /* spans alone */
    double co_a_ns, co_b_ns;             /* spans under co-run */
    double seq_ns;                       /* solo_a_ns + solo_b_ns: back to back */
    double col_ns;                       /* co-run makespan: last end - first start */
    int32_t overlapped;                  /* 1 if the two co-run spans intersect */
    int32_t status;                      /* first non-OK status of the four runs, else IFR_OK */
} ifr_pair_result;

/* Errors: IFR_ERR_ARG (null pointer, max_rounds <= 0, IFR_S_SCHED, invalid
 * configuration as in ifr_stressor_launch), IFR_ERR_CAPACITY (fewer than two free
 * stressor slots), IFR_ERR_TIMEOUT (a run did not finish within 60 s on the host),
 * IFR_ERR_CUDA.  A run whose blocks hit their deadline is reported in `status`. */
int ifr_stressor_pair(ifr_ctx *ctx, const ifr_stressor_cfg *a, const ifr_stressor_cfg *b, ifr_pair_result *out);

/* ---- a victim beside a fixed-work stressor, latency from release (Sec. 4.2) -- */
/* The paper's block-scheduler experiment launches a sleep kernel and an LLM decode
 * step together and reports the step's latency: a victim block that cannot fit next
 * to the sleeping blocks waits for them to leave (head-of-line blocking).  Because
 * such a victim starts late, its latency is counted from its release, not from its
 * first block.  ifr_colocate runs the victim's K launches alone, the stressor (fixed
 * work, max_rounds > 0, not IFR_S_SCHED) alone, and then the victim arriving at the
 * running stressor: both streams leave a device-side gate together, the victim's
 * stream waits (bounded, 200 ms) until every stressor block is resident, stamps its
 * release and launches.  Alone, the release is the gate's end.  *_ns = last block
 * exit - release (the stressor's from the gate). */
typedef struct {
    ifr_timing victim_solo, victim_co;        /* K victim launches alone / beside the stressor */
    ifr_stressor_result stress_solo, stress_co;
    double victim_solo_ns, victim_co_ns;      /* release to the victim's last block exit */
    double stress_solo_ns, stress_co_ns;      /* release to the stressor's last block exit */
    int32_t blocked;    /* 1 if no victim block started before a stressor block ended (left its SM) */
    int32_t status;     /* first non-OK status of the four runs, else IFR_OK */
} ifr_colocate_result;

/* Errors: IFR_ERR_ARG (null pointer, max_rounds <= 0, IFR_S_SCHED, invalid
 * configurations), IFR_ERR_CAPACITY, IFR_ERR_TIMEOUT (60 s host bound), IFR_ERR_CUDA. */
int ifr_colocate(ifr_ctx *ctx, const ifr_stressor_cfg *stressor, const ifr_victim_cfg *victim,
                 ifr_colocate_result *out);

/* ---- solo kernel profiles (Sec. 2.2 metrics; Sec. 5.1 estimator inputs) -- */
/* Static launch properties of the kernel a victim or stressor configuration
 * would run, the inputs of the SM-utilisation and occupancy metrics of Sec. 2.2
 * (threads, registers and shared memory per block decide how many blocks fit on an
 * SM, Sec. 2.1).  No GPU work is done. */
typedef struct {
    int32_t grid, block;           /* blocks per launch and threads per block */
    int32_t regs_per_thread;       /* registers per thread (cudaFuncGetAttributes) */
    int32_t static_smem;           /* bytes of static shared memory per block */
    int32_t dynamic_smem;          /* bytes of dynamic shared memory per block */
    int32_t max_blocks_per_sm;     /* occupancy limit of this launch shape */
    int32_t tmem_cols;             /* tensor-memory columns per block */
    int32_t uses_tensor;           /* 1 for tcgen05 kernels */
    int32_t sm_count;              /* stressors: SMs allowed; victims: 0 (all) */
    int32_t blocks_per_sm;         /* stressors: working blocks per allowed SM; victims: 0 */
    int32_t launches;              /* launches per measurement (victims: K; scheduler: chain) */
    int32_t reserved;
    double bytes_per_launch;       /* victims: algorithmic bytes of one launch (stressors: 0) */
    double flops_per_launch;       /* victims: algorithmic flops of one launch (stressors: 0) */
} ifr_kernel_profile;

/* Errors: IFR_ERR_ARG (invalid configuration, as in the launch calls), IFR_ERR_CUDA. */
int ifr_victim_profile(ifr_ctx *ctx, const ifr_victim_cfg *cfg, ifr_kernel_profile *out);
int ifr_stressor_profile(ifr_ctx *ctx, const ifr_stressor_cfg *cfg, ifr_kernel_profile *out);

/* ---- slowdown predictor (Sec. 5.1 kernel-level interference estimator) --- */
/* A multilayer perceptron on the solo profiles of a victim and a co-runner that
 * predicts the victim's log slowdown.  Layer l computes Z_l = H_l W_l^T + b_l
 * (bf16 operands, fp32 accumulation) and, for hidden layers, H_{l+1} =
 * bf16(GELU(Z_l)) with the exact erf GELU; the last layer has one output.
 * All buffers are caller-owned device memory, row-major; nothing is allocated. */
#define IFR_MLP_MAX_LAYERS 8
typedef struct {
    int32_t n_layers;                     /* 1..IFR_MLP_MAX_LAYERS */
    int32_t batch;                        /* rows B */
    int32_t dims[IFR_MLP_MAX_LAYERS + 1]; /* dims[0] inputs ... dims[n_layers] = 1 */
    const void *W[IFR_MLP_MAX_LAYERS];    /* bf16 [dims[l+1]][dims[l]] */
    const float *b[IFR_MLP_MAX_LAYERS];   /* fp32 [dims[l+1]] */
    void *H[IFR_MLP_MAX_LAYERS];          /* bf16 [B][dims[l]]; H[0] is the input X */
    float *Z[IFR_MLP_MAX_LAYERS];         /* fp32 [B][dims[l+1]] pre-activations (forward output) */
    float *dW[IFR_MLP_MAX_LAYERS];        /* fp32 [dims[l+1]][dims[l]] (backward output) */
    float *db[IFR_MLP_MAX_LAYERS];        /* fp32 [dims[l+1]] (backward output) */
    float *dZ[IFR_MLP_MAX_LAYERS];        /* fp32 [B][dims[l+1]] backward workspace */
    void *dZh[IFR_MLP_MAX_LAYERS];        /* bf16 [B][dims[l+1]] backward workspace */
    float *dX;                            /* fp32 [B][dims[0]] input gradient, or NULL */
} ifr_mlp;

/* Forward pass on `stream` (cudaStream_t; NULL = legacy default).  Writes Z[l]
 * for every layer and H[l+1] for hidden layers; the prediction is Z[n_layers-1]
 * ([B][1]).  Errors: IFR_ERR_ARG (shape, null buffer, last dim != 1), IFR_ERR_CUDA. */
int ifr_mlp_forward(ifr_ctx *ctx, const ifr_mlp *mlp, void *stream);
/* Backward pass for dY = dLoss/dprediction ([B] fp32): writes dW, db for every
 * layer and dX when non-NULL.  GEMM operands are bf16 (dZ rounded once), the bias
 * gradient uses the fp32 dZ.  Needs the Z and H of the matching forward pass. */
int ifr_mlp_backward(ifr_ctx *ctx, const ifr_mlp *mlp, const float *dY, void *stream);
/* Mean-squared error of yhat against target (n <= any): dY = 2 (yhat - t) / n and
 * *loss = mean((yhat - t)^2) (loss may be NULL); device pointers. */
int ifr_mse_grad(ifr_ctx *ctx, const float *yhat, const float *target, int n, float *dY, float *loss,
                 void *stream);
/* One Adam step (Kingma & Ba 2015; eps added after the square root, no weight
 * decay) over n fp32 parameters w with gradient g and moments m, v (all device);
 * `step` is 1-based; when w_bf16 is non-NULL the updated weights are also stored
 * there as bf16. */
int ifr_adam_step(ifr_ctx *ctx, float *w, const float *g, float *m, float *v, void *w_bf16, int64_t n, float lr,
                  float beta1, float beta2, float eps, int step, void *stream);

/* ---- sweep (Sec. 4.1 method) -------------------------------------------- */
typedef struct {
    int32_t n_victims;
    const ifr_victim_cfg *victims;
    int32_t n_stressors;
    int32_t n_levels;                    /* levels 1..L per stressor (level 0 is added) */
    const ifr_stressor_cfg *levels;      /* [n_stressors][n_levels] full configurations */
    int32_t repeats;                     /* measurements per cell */
    int32_t batched;                     /* 0: launch per cell; 1: one captured CUDA graph
                                            per (stressor, level) over all victims, each
                                            victim its own launches; 2: the same graphs
                                            with grouped persistent victims:
                                            layernorm and softmax victims of one row
                                            template, GEMV victims of more than 256
                                            columns, and variant-0 GEMMs of one tile
                                            width run as one launch per group (at most
                                            16) whose walkers claim rows or tiles in
                                            order and start a victim only after the
                                            previous one has finished, each victim
                                            timed on its own; other victims run alone.
                                            Walkers that claim work on demand make the
                                            victims less sensitive than their own
                                            launches (mode 1 is the measurement mode).
                                            Other values: IFR_ERR_ARG */
} ifr_sweep_plan;

typedef struct {
    int32_t victim, stressor, level, repeat; /* stressor -1 = solo; level 0 = zero-SM stressor */
    ifr_timing timing;
    ifr_stressor_result stress;               /* zeroed for solo cells */
    int32_t valid;                            /* constant-interference rule met (Sec. 4.1) */
    int32_t status;
} ifr_cell_result;

/* Run the plan: per repeat, solo runs of every victim, then for every stressor
 * and level 0..L a colocated measurement of every victim.  Writes up to `cap`
 * cells in that order and sets *n_out.  Errors: IFR_ERR_ARG, IFR_ERR_CAPACITY,
 * IFR_ERR_CUDA.  A cell whose stressor timed out is recorded with valid = 0.  In the
 * plain sweep (batched = 0), a scheduler-stressor cell whose chain of launches ended
 * before the victim did (the rule's only failure) is measured again with four times
 * the launches, at most three times and up to 16384 launches (a chain already that
 * long is not measured again); the cell keeps the last measurement. */
int ifr_sweep(ifr_ctx *ctx, const ifr_sweep_plan *plan, ifr_cell_result *cells, size_t cap, size_t *n_out);

/* ---- kernel-with-kernel colocation (Sec. 4.1; Table 3 seq/col speedup) ---- */
typedef struct {
    ifr_timing victim_solo;     /* victim alone, K launches */
    ifr_timing corunner_solo;   /* co-runner alone, one launch */
    ifr_timing victim_corun;    /* victim while the co-runner chain runs */
    ifr_timing corunner_corun;  /* the co-runner chain during the co-run */
    int32_t valid;              /* the chain's first block started before the victim's first
                                   block and its last block ended after the victim's last */
    int32_t status;
    int32_t corunner_launches;  /* length of the co-runner chain */
    int32_t blocked;            /* head-of-line blocked (Sec. 4.2): no victim block could start
                                   before the whole co-runner chain had finished */
    uint64_t victim_release_ns; /* %globaltimer when the victim was released (a co-runner
                                   block was running); latency = victim end - release */
    double victim_slowdown;     /* (victim_corun span / K) / (victim_solo span / K), spans =
                                   last block exit - first block entry (Sec. 4.3 slowdown);
                                   NaN when a span is empty */
    double corunner_slowdown;   /* the same for the co-runner chain: its per-launch time during
                                   the co-run over its solo launch time */
} ifr_corun_result;

/* Colocate two workloads on concurrent streams: the co-runner runs as a chain of
 * back-to-back launches on the context's stressor stream (long enough to cover
 * 4x the victim's solo window when corunner_launches = 0), the victim's K
 * launches start on the victim stream once a co-runner block is running (bounded
 * wait), and every launch stamps %globaltimer.  The call reduces the raw stamps
 * to victim_slowdown = (victim_corun span / K) / (victim_solo span / K) and the
 * co-runner's slowdown likewise (Sec. 4.3, 4.4.1).  Both configurations are
 * validated as in ifr_victim_launch.  Errors: IFR_ERR_ARG, IFR_ERR_CUDA,
 * IFR_ERR_TIMEOUT (host wait). */
int ifr_corun(ifr_ctx *ctx, const ifr_victim_cfg *victim, const ifr_victim_cfg *corunner, int corunner_launches,
              ifr_corun_result *out);

/* ---- sensitivity reduction (Sec. 4.3 slowdown; Sec. 5.1 estimator input) - */
typedef struct {
    int32_t n_stressors, n_levels;
    double t0_ns;                                       /* median solo duration per launch */
    double noise;                                       /* (max-min)/median of solo */
    double slowdown[IFR_MAX_STRESSORS][IFR_MAX_LEVELS + 1]; /* NaN where no valid cell */
    double S[IFR_MAX_STRESSORS];                        /* slowdown at level L minus 1 */
    double auc[IFR_MAX_STRESSORS];                      /* trapezoid of slowdown-1 over x */
    int32_t monotone[IFR_MAX_STRESSORS];
    int32_t n_valid, n_invalid;
} ifr_sensitivity_out;

/* Pure host reduction of one victim's cells (see the oracle's reduction for the
 * exact rule).  intensity: [n_stressors][n_levels] achieved fraction x_l of each
 * level, or NULL for x_l = l / n_levels.  Errors: IFR_ERR_ARG. */
int ifr_sensitivity(const ifr_cell_result *cells, size_t n, int victim, int n_stressors, int n_levels,
                    const double *intensity, ifr_sensitivity_out *out);

#ifdef __cplusplus
}
#endif
#endif /* IFR_H */
