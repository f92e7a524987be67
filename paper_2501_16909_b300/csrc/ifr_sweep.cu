// Colocation sweep (Sec. 4.1): a stressor holding a constant interference level on
// one stream, victims on another, slowdown against isolated runs.
//
// Plain mode, per colocated cell:
//   stressor stream:  reset state -> stressor kernels
//   victim stream:    reset timing -> bounded residency wait -> K victim launches
//                     -> stop flag (copy-engine write, so it needs no SM slot)
// Batched mode, per (stressor, level): the same sequence with all victims
// back to back under one stressor run, captured once into a CUDA graph and
// replayed for every repeat; per-victim timings land in separate slots.  Grouped
// batched mode: the same graphs, with victims of one kernel run as one persistent
// grouped launch that walks their rows or tiles in order (ifr_victims_enqueue_group).
#include <math.h>
#include <string.h>
#include <time.h>

#include <vector>

#include "ifr_internal.cuh"

namespace {

constexpr uint64_t kResidencyTimeoutNs = 200000000ull;  // 200 ms
constexpr int kSchedRetryMaxLaunches = 16384;              // longest scheduler chain of a re-measured cell

int wait_event_bounded(cudaEvent_t ev, int timeout_ms) {
    int waited_us = 0;
    cudaError_t q;
    while ((q = cudaEventQuery(ev)) == cudaErrorNotReady) {
        if (waited_us >= timeout_ms * 1000) return IFR_ERR_TIMEOUT;
        struct timespec ts = {0, 20000};
        nanosleep(&ts, nullptr);
        waited_us += 20;
    }
    if (q != cudaSuccess) return ifr_cuda_fail(q, "cudaEventQuery", __FILE__, __LINE__);
    return IFR_OK;
}

// A scheduler chain is a fixed number of launches.  One that ended before the
// victim did (no recorded block saw the stop request, which follows the victim)
// fails the constant-interference rule at the end only.
bool sched_chain_short(const ifr_stressor_cfg &sc, const ifr_cell_result &c) {
    const ifr_timing &t = c.timing;
    const ifr_stressor_result &s = c.stress;
    return sc.kind == IFR_S_SCHED && c.level > 0 && !c.valid && t.status == IFR_OK && s.status == IFR_OK &&
           s.blocks_active > 0 && s.t_start_last_ns <= t.t_start_ns && s.t_end_first_ns < t.t_end_ns;
}

void fill_validity(ifr_cell_result &c) {
    const ifr_timing &t = c.timing;
    const ifr_stressor_result &s = c.stress;
    int ok = t.status == IFR_OK && t.t_end_ns > t.t_start_ns;
    if (ok && c.stressor >= 0) {
        ok = s.status == IFR_OK;
        if (ok && c.level > 0)
            ok = s.blocks_active > 0 && s.t_start_last_ns <= t.t_start_ns && s.t_end_first_ns >= t.t_end_ns;
    }
    c.valid = ok;
    c.status = ok ? IFR_OK : (t.status != IFR_OK ? t.status : (s.status != IFR_OK ? s.status : IFR_ERR_INVALID_CELL));
}

ifr_stressor_cfg level_cfg(const ifr_sweep_plan *p, int r, int l) {
    ifr_stressor_cfg c = p->levels[(size_t)r * p->n_levels + (l > 0 ? l - 1 : 0)];
    if (l == 0) c.sm_count = 0;  // level 0: the harness runs, nothing interferes
    return c;
}

int measure_solo_plain(ifr_ctx *ctx, const ifr_victim_cfg *v, ifr_timing *out) {
    DevTiming *tm = ctx->d_timing;
    cudaStream_t sv = ctx->s_victim;
    int rc = ifr_timing_reset(tm, 1, sv, nullptr);
    if (rc) return rc;
    ctx->kernel_launches += 1;
    IFR_CUDA(cudaEventRecord(ctx->ev_a, sv));
    rc = ifr_victim_enqueue(ctx, v, sv, tm);
    if (rc) return rc;
    IFR_CUDA(cudaEventRecord(ctx->ev_b, sv));
    rc = wait_event_bounded(ctx->ev_b, 60000);
    if (rc) return rc;
    DevTiming h;
    IFR_CUDA(cudaMemcpy(&h, tm, sizeof h, cudaMemcpyDeviceToHost));
    ifr_timing_to_host(h, v->repeats > 0 ? v->repeats : 1, out);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev_a, ctx->ev_b);
    out->event_ms = ms;
    return IFR_OK;
}

int measure_cell_plain(ifr_ctx *ctx, const ifr_victim_cfg *v, const ifr_stressor_cfg *scfg, ifr_cell_result *cell) {
    int slot = ifr_slot_alloc(ctx);
    if (slot < 0) return slot;
    cudaStream_t ss = ctx->s_stress, sv = ctx->s_victim;
    DevTiming *tm = ctx->d_timing;
    ctx->slots[slot].watch = 1;
    int rc = ifr_stressor_enqueue(ctx, scfg, ss, slot);
    if (rc) return rc;
    rc = ifr_timing_reset(tm, 1, sv, ctx->d_progress);
    ctx->kernel_launches += 1;
    if (!rc) rc = ifr_enqueue_wait_resident(ctx, slot, sv, tm, kResidencyTimeoutNs);
    if (!rc) {
        cudaEventRecord(ctx->ev_a, sv);
        rc = ifr_victim_enqueue(ctx, v, sv, tm);
        cudaEventRecord(ctx->ev_b, sv);
    }
    int rc_stop = ifr_enqueue_stop(ctx, slot, sv);
    if (!rc) rc = rc_stop;
    int rc_w = wait_event_bounded(ctx->ev_b, 60000);
    ifr_stressor_result sres;
    int rc_s = ifr_stressor_wait(ctx, slot, 60000, &sres);
    ctx->slots[slot].in_use = 0;
    if (rc) return rc;
    if (rc_w) return rc_w;
    DevTiming h;
    IFR_CUDA(cudaMemcpy(&h, tm, sizeof h, cudaMemcpyDeviceToHost));
    ifr_timing_to_host(h, v->repeats > 0 ? v->repeats : 1, &cell->timing);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev_a, ctx->ev_b);
    cell->timing.event_ms = ms;
    cell->stress = sres;
    if (rc_s == IFR_ERR_TIMEOUT && cell->stress.status == IFR_OK) cell->stress.status = IFR_ERR_TIMEOUT;
    else if (rc_s) return rc_s;
    return IFR_OK;
}

// The victims of a grouped batch: victims with the same grouping key and launch count
// run as one grouped launch (at most IFR_GROUP_MAX victims each), placed where the
// first of them stands in the plan; the others run alone, in plan order.  Each victim
// keeps its own measurement record.
int enqueue_victims_grouped(ifr_ctx *ctx, const ifr_sweep_plan *p, cudaStream_t sv) {
    const int nv = p->n_victims;
    std::vector<int> key((size_t)nv), done((size_t)nv, 0);
    for (int v = 0; v < nv; ++v) key[v] = ifr_victim_group_key(ctx, &p->victims[v]);
    auto reps = [&](int v) { return p->victims[v].repeats > 0 ? p->victims[v].repeats : 1; };
    for (int v = 0; v < nv; ++v) {
        if (done[v]) continue;
        done[v] = 1;
        int rc;
        if (key[v] <= 0) {
            rc = ifr_victim_enqueue(ctx, &p->victims[v], sv, ctx->d_timing + v);
        } else {
            std::vector<const ifr_victim_cfg *> vs(1, &p->victims[v]);
            std::vector<DevTiming *> tms(1, ctx->d_timing + v);
            for (int w = v + 1; w < nv && (int)vs.size() < IFR_GROUP_MAX; ++w)
                if (!done[w] && key[w] == key[v] && reps(w) == reps(v)) {
                    done[w] = 1;
                    vs.push_back(&p->victims[w]);
                    tms.push_back(ctx->d_timing + w);
                }
            rc = ifr_victims_enqueue_group(ctx, vs.data(), tms.data(), (int)vs.size(), sv);
        }
        if (rc) return rc;
    }
    return IFR_OK;
}

// Capture one graph: optional stressor + all victims back to back (grouped when the
// plan asks for it).
int capture_batch(ifr_ctx *ctx, const ifr_sweep_plan *p, const ifr_stressor_cfg *scfg, int slot,
                  cudaGraphExec_t *exec, uint64_t *kernels) {
    const uint64_t before = ctx->kernel_launches;
    cudaStream_t sv = ctx->s_victim, ss = ctx->s_stress;
    cudaGraph_t g = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    IFR_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    IFR_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    int rc = IFR_OK;
    IFR_CUDA(cudaStreamBeginCapture(sv, cudaStreamCaptureModeRelaxed));
    rc = ifr_timing_reset(ctx->d_timing, p->n_victims, sv, scfg ? ctx->d_progress : nullptr);
    ctx->kernel_launches += 1;
    if (!rc && scfg) {
        cudaEventRecord(fork, sv);
        cudaStreamWaitEvent(ss, fork, 0);
        rc = ifr_stressor_enqueue(ctx, scfg, ss, slot, 0);
        if (!rc) rc = ifr_enqueue_wait_resident(ctx, slot, sv, ctx->d_timing, kResidencyTimeoutNs);
    }
    if (!rc && p->batched == 2)
        rc = enqueue_victims_grouped(ctx, p, sv);
    else
        for (int v = 0; !rc && v < p->n_victims; ++v)
            rc = ifr_victim_enqueue(ctx, &p->victims[v], sv, ctx->d_timing + v);
    if (!rc && scfg) {
        rc = ifr_enqueue_stop(ctx, slot, sv);
        cudaEventRecord(join, ss);
        cudaStreamWaitEvent(sv, join, 0);
    }
    cudaError_t e = cudaStreamEndCapture(sv, &g);
    if (!rc && e != cudaSuccess) rc = ifr_cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    if (!rc) {
        e = cudaGraphInstantiate(exec, g, 0);
        if (e != cudaSuccess) rc = ifr_cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
    if (g) cudaGraphDestroy(g);
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
    *kernels = ctx->kernel_launches - before;
    ctx->kernel_launches = before;  // counted again at every replay
    return rc;
}

// Waits (bounded) until a block of the measurement `tm` has started, then
// stamps the release time into *release.
__global__ void wait_started_kernel(const DevTiming *tm, uint64_t timeout_ns, DevTiming *status_to,
                                    uint64_t *release) {
    if (threadIdx.x != 0) return;
    const uint64_t t0 = ifr_gtimer();
    uint32_t it = 0;
    while (*(const volatile uint64_t *)&tm->t_min == ~0ull) {
        if (ifr_gtimer() - t0 > timeout_ns || ++it > (1u << 22)) {
            status_to->status = IFR_ERR_NOT_RESIDENT;
            break;
        }
        __nanosleep(256);
    }
    *release = ifr_gtimer();
}

int read_timing(ifr_ctx *ctx, int slot, int repeats, ifr_timing *out) {
    DevTiming h;
    IFR_CUDA(cudaMemcpy(&h, ctx->d_timing + slot, sizeof h, cudaMemcpyDeviceToHost));
    ifr_timing_to_host(h, repeats, out);
    return IFR_OK;
}

// Slowdown of one measurement against another (Sec. 4.3: colocated over isolated
// latency), each as (last block exit - first block entry) / K; NaN without a span.
double per_launch_ratio(const ifr_timing &co, const ifr_timing &solo) {
    const double kc = co.repeats > 0 ? co.repeats : 1, ks = solo.repeats > 0 ? solo.repeats : 1;
    if (co.t_end_ns <= co.t_start_ns || solo.t_end_ns <= solo.t_start_ns) return NAN;
    return (((double)co.t_end_ns - (double)co.t_start_ns) / kc) / (((double)solo.t_end_ns - (double)solo.t_start_ns) / ks);
}

// The CTA-pair GEMM (variant 2) allocates the same TMEM columns on two SMs at once,
// and the two-accumulator GEMMs (variants 3, 4) all 512 columns of an SM; beside other
// TMEM users (the tensor stressor, another GEMM) those allocations can wait until
// they exit, so the measurements that colocate kernels refuse both.  The bulk-copy
// GEMV (variant 1) is a solo variant too: its 80 KiB of shared memory per block is
// not in the co-residence budget the stressors leave room for.
int colocatable(const ifr_victim_cfg *c) {
    if (c->kind == IFR_V_GEMM && c->variant >= 2) return IFR_ERR_ARG;
    if (c->kind == IFR_V_GEMV && c->variant == 1) return IFR_ERR_ARG;
    return IFR_OK;
}

}  // namespace

extern "C" int ifr_corun(ifr_ctx *ctx, const ifr_victim_cfg *victim, const ifr_victim_cfg *corunner,
                         int corunner_launches, ifr_corun_result *out) {
    if (!ctx || !out || corunner_launches < 0 || corunner_launches > 100000) return IFR_ERR_ARG;
    int rc = ifr_victim_validate(ctx, victim);
    if (!rc) rc = ifr_victim_validate(ctx, corunner);
    if (!rc) rc = colocatable(victim);
    if (!rc) rc = colocatable(corunner);
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    rc = ifr_ensure_timing(ctx, 3);
    if (rc) return rc;
    IFR_CUDA(cudaDeviceSynchronize());
    cudaStream_t sv = ctx->s_victim, ss = ctx->s_stress;
    const int Kv = victim->repeats > 0 ? victim->repeats : 1;
    // solo runs
    rc = measure_solo_plain(ctx, victim, &out->victim_solo);
    if (rc) return rc;
    ifr_victim_cfg one = *corunner;
    one.repeats = 1;
    rc = measure_solo_plain(ctx, &one, &out->corunner_solo);
    if (rc) return rc;
    int n = corunner_launches;
    if (n == 0) {
        const double tv = (double)(out->victim_solo.t_end_ns - out->victim_solo.t_start_ns);
        const double tc = (double)(out->corunner_solo.t_end_ns - out->corunner_solo.t_start_ns);
        n = (int)(4.0 * tv / (tc > 1.0 ? tc : 1.0)) + 2;
        if (n > 20000) n = 20000;
    }
    out->corunner_launches = n;
    one.repeats = n;
    // co-run: chain on the stressor stream, victim once a chain block is running
    DevTiming *tv = ctx->d_timing, *tc = ctx->d_timing + 1;
    cudaEvent_t reset_done;
    IFR_CUDA(cudaEventCreateWithFlags(&reset_done, cudaEventDisableTiming));
    // The victim side (waiter + K launches) is enqueued before the chain, so the
    // waiter is already pending on the GPU when the chain's first block starts.
    rc = ifr_timing_reset(tc, 1, ss, nullptr);
    cudaEventRecord(reset_done, ss);
    if (!rc) rc = ifr_timing_reset(tv, 1, sv, nullptr);
    cudaStreamWaitEvent(sv, reset_done, 0);
    uint64_t *release = (uint64_t *)(ctx->d_timing + 2);  // scratch word past the two measurements
    if (!rc) {
        wait_started_kernel<<<1, 32, 0, sv>>>(tc, 200000000ull, tv, release);
        ctx->kernel_launches += 3;
        rc = ifr_victim_enqueue(ctx, victim, sv, tv);
    }
    if (!rc) rc = ifr_victim_enqueue(ctx, &one, ss, tc);
    IFR_CUDA(cudaEventRecord(ctx->ev_b, sv));
    IFR_CUDA(cudaEventRecord(ctx->ev_a, ss));
    int rc1 = wait_event_bounded(ctx->ev_b, 120000);
    int rc2 = wait_event_bounded(ctx->ev_a, 120000);
    cudaEventDestroy(reset_done);
    if (rc) return rc;
    if (rc1) return rc1;
    if (rc2) return rc2;
    rc = read_timing(ctx, 0, Kv, &out->victim_corun);
    if (!rc) rc = read_timing(ctx, 1, n, &out->corunner_corun);
    if (rc) return rc;
    IFR_CUDA(cudaMemcpy(&out->victim_release_ns, release, sizeof(uint64_t), cudaMemcpyDeviceToHost));
    const ifr_timing &a = out->victim_corun, &b = out->corunner_corun;
    out->victim_slowdown = per_launch_ratio(out->victim_corun, out->victim_solo);
    out->corunner_slowdown = per_launch_ratio(out->corunner_corun, out->corunner_solo);
    out->valid = a.status == IFR_OK && b.status == IFR_OK && b.t_start_ns <= a.t_start_ns && b.t_end_ns >= a.t_end_ns;
    out->blocked = a.status == IFR_OK && a.t_start_ns >= b.t_end_ns;
    out->status = a.status != IFR_OK ? a.status : (out->valid ? IFR_OK : (out->blocked ? IFR_ERR_HOL : IFR_ERR_INVALID_CELL));
    return IFR_OK;
}

namespace {
// Holds its stream for `ns` of %globaltimer (bounded), so that work enqueued on
// other streams behind an event recorded after it is released at one instant;
// stamps the release time into *release when given.
__global__ void gate_kernel(uint64_t ns, uint64_t *release) {
    if (threadIdx.x != 0) return;
    const uint64_t t0 = ifr_gtimer();
    uint32_t it = 0;
    while (ifr_gtimer() - t0 < ns && ++it < (1u << 22)) __nanosleep(1000);
    if (release) *release = ifr_gtimer();
}

// Stamps %globaltimer into *release (the point from which a victim's latency counts).
__global__ void stamp_kernel(uint64_t *release) {
    if (threadIdx.x == 0) *release = ifr_gtimer();
}

// Enqueue the gate on the control stream and make `a` (and `b`, if given) wait for it.
int enqueue_gate(ifr_ctx *ctx, cudaStream_t a, cudaStream_t b, uint64_t *release) {
    ifr_carveout((const void *)gate_kernel);
    gate_kernel<<<1, 32, 0, ctx->s_ctrl>>>(300000ull, release);
    IFR_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    IFR_CUDA(cudaEventRecord(ctx->ev_a, ctx->s_ctrl));
    IFR_CUDA(cudaStreamWaitEvent(a, ctx->ev_a, 0));
    if (b) IFR_CUDA(cudaStreamWaitEvent(b, ctx->ev_a, 0));
    return IFR_OK;
}

double span_ns(const ifr_stressor_result &r) {
    return r.t_end_ns > r.t_start_ns ? (double)(r.t_end_ns - r.t_start_ns) : 0.0;
}

// One fixed-work stressor run on `stream` in a fresh slot; fills *out.
int run_fixed(ifr_ctx *ctx, const ifr_stressor_cfg *cfg, cudaStream_t stream, ifr_stressor_result *out) {
    const int slot = ifr_slot_alloc(ctx);
    if (slot < 0) return slot;
    ctx->slots[slot].watch = 0;
    int rc = ifr_stressor_enqueue(ctx, cfg, stream, slot);
    if (rc) return rc;
    rc = wait_event_bounded(ctx->slots[slot].ev_end, 60000);
    if (!rc) rc = ifr_stressor_collect(ctx, slot);
    if (!rc) *out = ctx->slots[slot].result;
    ctx->slots[slot].in_use = 0;
    return rc;
}
}  // namespace

extern "C" int ifr_stressor_pair(ifr_ctx *ctx, const ifr_stressor_cfg *a, const ifr_stressor_cfg *b,
                                 ifr_pair_result *out) {
    if (!ctx || !a || !b || !out) return IFR_ERR_ARG;
    if (a->max_rounds <= 0 || b->max_rounds <= 0 || a->kind == IFR_S_SCHED || b->kind == IFR_S_SCHED)
        return IFR_ERR_ARG;
    memset(out, 0, sizeof *out);
    IFR_CUDA(cudaDeviceSynchronize());
    // each alone on the stream it co-runs on (under ifr_partition: its own partition)
    int rc = run_fixed(ctx, a, ctx->s_stress, &out->solo_a);
    if (!rc) rc = run_fixed(ctx, b, ctx->s_victim, &out->solo_b);
    if (rc) return rc;
    // co-run: both streams wait behind a 300 us gate, then run their reset and kernel
    const int sa = ifr_slot_alloc(ctx);
    if (sa < 0) return sa;
    ctx->slots[sa].watch = 0;
    ctx->slots[sa].in_use = 1;  // reserve while the second slot is chosen
    const int sb = ifr_slot_alloc(ctx);
    ctx->slots[sa].in_use = 0;
    if (sb < 0) return sb;
    ctx->slots[sb].watch = 0;
    rc = enqueue_gate(ctx, ctx->s_stress, ctx->s_victim, nullptr);
    if (rc) return rc;
    rc = ifr_stressor_enqueue(ctx, a, ctx->s_stress, sa);
    if (rc) return rc;
    rc = ifr_stressor_enqueue(ctx, b, ctx->s_victim, sb);
    if (rc) {
        wait_event_bounded(ctx->slots[sa].ev_end, 60000);
        ctx->slots[sa].in_use = 0;
        return rc;
    }
    int rc1 = wait_event_bounded(ctx->slots[sa].ev_end, 60000);
    int rc2 = wait_event_bounded(ctx->slots[sb].ev_end, 60000);
    if (!rc1) rc1 = ifr_stressor_collect(ctx, sa);
    if (!rc2) rc2 = ifr_stressor_collect(ctx, sb);
    out->co_a = ctx->slots[sa].result;
    out->co_b = ctx->slots[sb].result;
    ctx->slots[sa].in_use = 0;
    ctx->slots[sb].in_use = 0;
    if (rc1) return rc1;
    if (rc2) return rc2;
    out->solo_a_ns = span_ns(out->solo_a);
    out->solo_b_ns = span_ns(out->solo_b);
    out->co_a_ns = span_ns(out->co_a);
    out->co_b_ns = span_ns(out->co_b);
    out->seq_ns = out->solo_a_ns + out->solo_b_ns;
    const uint64_t t0 = out->co_a.t_start_ns < out->co_b.t_start_ns ? out->co_a.t_start_ns : out->co_b.t_start_ns;
    const uint64_t t1 = out->co_a.t_end_ns > out->co_b.t_end_ns ? out->co_a.t_end_ns : out->co_b.t_end_ns;
    out->col_ns = t1 > t0 ? (double)(t1 - t0) : 0.0;
    out->overlapped = out->co_a.t_start_ns < out->co_b.t_end_ns && out->co_b.t_start_ns < out->co_a.t_end_ns;
    const int32_t sts[4] = {out->solo_a.status, out->solo_b.status, out->co_a.status, out->co_b.status};
    out->status = IFR_OK;
    for (int i = 0; i < 4; ++i)
        if (sts[i] != IFR_OK) {
            out->status = sts[i];
            break;
        }
    return IFR_OK;
}

extern "C" int ifr_colocate(ifr_ctx *ctx, const ifr_stressor_cfg *sc, const ifr_victim_cfg *vc,
                            ifr_colocate_result *out) {
    if (!ctx || !sc || !vc || !out) return IFR_ERR_ARG;
    if (sc->max_rounds <= 0 || sc->kind == IFR_S_SCHED) return IFR_ERR_ARG;
    int rc = ifr_victim_validate(ctx, vc);
    if (!rc) rc = colocatable(vc);
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    rc = ifr_ensure_timing(ctx, 3);
    if (rc) return rc;
    IFR_CUDA(cudaDeviceSynchronize());
    const int K = vc->repeats > 0 ? vc->repeats : 1;
    DevTiming *tv = ctx->d_timing;
    // scratch words past the measurements: gate end, victim release (co-run)
    uint64_t *gate_t = (uint64_t *)(ctx->d_timing + 2), *vrel = gate_t + 1;
    // mode 0: victim alone, 1: stressor alone, 2: victim arriving at the running stressor
    for (int mode = 0; mode < 3; ++mode) {
        const bool run_v = mode != 1, run_s = mode != 0;
        if (run_v) {
            rc = ifr_timing_reset(tv, 1, ctx->s_victim, nullptr);
            if (rc) return rc;
        }
        rc = enqueue_gate(ctx, ctx->s_victim, ctx->s_stress, gate_t);
        if (rc) return rc;
        int slot = -1;
        if (run_s) {
            slot = ifr_slot_alloc(ctx);
            if (slot < 0) return slot;
            ctx->slots[slot].watch = 0;
            rc = ifr_stressor_enqueue(ctx, sc, ctx->s_stress, slot);
            if (rc) return rc;
        }
        if (run_v && run_s) {
            // the victim arrives at a running stressor: every stressor block resident
            // first (bounded wait, 200 ms), then the release stamp.  A failure from here
            // on still waits for the enqueued stressor and frees its slot below.
            rc = ifr_enqueue_wait_resident(ctx, slot, ctx->s_victim, tv, 200000000ull);
            if (!rc) {
                ifr_carveout((const void *)stamp_kernel);
                stamp_kernel<<<1, 32, 0, ctx->s_victim>>>(vrel);
                const cudaError_t e = cudaGetLastError();
                rc = e == cudaSuccess ? IFR_OK : ifr_cuda_fail(e, "stamp_kernel", __FILE__, __LINE__);
                ctx->kernel_launches += 1;
            }
        }
        if (run_v && !rc) {
            rc = ifr_victim_enqueue(ctx, vc, ctx->s_victim, tv);
            if (!rc) rc = cudaEventRecord(ctx->ev_b, ctx->s_victim) == cudaSuccess ? IFR_OK : IFR_ERR_CUDA;
        }
        int rcv = run_v && !rc ? wait_event_bounded(ctx->ev_b, 60000) : IFR_OK;
        int rcs = run_s ? wait_event_bounded(ctx->slots[slot].ev_end, 60000) : IFR_OK;
        if (run_s && !rcs) rcs = ifr_stressor_collect(ctx, slot);
        if (run_s) ctx->slots[slot].in_use = 0;
        if (rc) return rc;
        if (rcv) return rcv;
        if (rcs) return rcs;
        uint64_t stamps[2] = {0, 0};
        IFR_CUDA(cudaMemcpy(stamps, gate_t, sizeof stamps, cudaMemcpyDeviceToHost));
        const uint64_t rel = stamps[0], rel_v = run_s ? stamps[1] : stamps[0];
        ifr_timing t;
        memset(&t, 0, sizeof t);
        if (run_v) {
            rc = read_timing(ctx, 0, K, &t);
            if (rc) return rc;
        }
        const ifr_stressor_result r = run_s ? ctx->slots[slot].result : ifr_stressor_result{};
        const double tv_ns = run_v && t.t_end_ns > rel_v ? (double)(t.t_end_ns - rel_v) : 0.0;
        const double ts_ns = run_s && r.t_end_ns > rel ? (double)(r.t_end_ns - rel) : 0.0;
        if (mode == 0) {
            out->victim_solo = t;
            out->victim_solo_ns = tv_ns;
        } else if (mode == 1) {
            out->stress_solo = r;
            out->stress_solo_ns = ts_ns;
        } else {
            out->victim_co = t;
            out->stress_co = r;
            out->victim_co_ns = tv_ns;
            out->stress_co_ns = ts_ns;
        }
    }
    // blocked: no victim block could start until a stressor block had left its SM
    out->blocked = out->victim_co.t_start_ns >= out->stress_co.t_end_first_ns;
    const int32_t sts[4] = {out->victim_solo.status, out->stress_solo.status, out->victim_co.status,
                            out->stress_co.status};
    out->status = IFR_OK;
    for (int i = 0; i < 4; ++i)
        if (sts[i] != IFR_OK) {
            out->status = sts[i];
            break;
        }
    return IFR_OK;
}

extern "C" int ifr_sweep(ifr_ctx *ctx, const ifr_sweep_plan *p, ifr_cell_result *cells, size_t cap, size_t *n_out) {
    if (!ctx || !p || !n_out || p->n_victims <= 0 || !p->victims || p->n_stressors < 0 ||
        p->n_stressors > IFR_MAX_STRESSORS || p->n_levels < 0 || p->n_levels > IFR_MAX_LEVELS || p->repeats <= 0 ||
        p->batched < 0 || p->batched > 2)
        return IFR_ERR_ARG;
    if (p->n_stressors > 0 && (p->n_levels <= 0 || !p->levels)) return IFR_ERR_ARG;
    *n_out = 0;
    for (int v = 0; v < p->n_victims; ++v) {
        int rc = ifr_victim_validate(ctx, &p->victims[v]);
        if (!rc) rc = colocatable(&p->victims[v]);
        if (rc) return rc;
    }
    const size_t need = (size_t)p->repeats * p->n_victims * (1 + (size_t)p->n_stressors * (p->n_levels + 1));
    if (!cells || cap < need) return IFR_ERR_CAPACITY;
    int rc = ifr_ensure_timing(ctx, p->n_victims);
    if (rc) return rc;
    IFR_CUDA(cudaDeviceSynchronize());
    size_t n = 0;
    if (!p->batched) {
        for (int rep = 0; rep < p->repeats; ++rep) {
            for (int v = 0; v < p->n_victims; ++v) {
                ifr_cell_result &c = cells[n++];
                memset(&c, 0, sizeof c);
                c.victim = v;
                c.stressor = -1;
                c.repeat = rep;
                rc = measure_solo_plain(ctx, &p->victims[v], &c.timing);
                if (rc) return rc;
                fill_validity(c);
            }
            for (int r = 0; r < p->n_stressors; ++r)
                for (int l = 0; l <= p->n_levels; ++l) {
                    ifr_stressor_cfg sc = level_cfg(p, r, l);
                    for (int v = 0; v < p->n_victims; ++v) {
                        ifr_cell_result &c = cells[n++];
                        memset(&c, 0, sizeof c);
                        c.victim = v;
                        c.stressor = r;
                        c.level = l;
                        c.repeat = rep;
                        rc = measure_cell_plain(ctx, &p->victims[v], &sc, &c);
                        if (rc) return rc;
                        fill_validity(c);
                        // a chain too short for this victim: measure again with four
                        // times the launches, at most three times
                        ifr_stressor_cfg longer = sc;
                        for (int retry = 0; retry < 3 && sched_chain_short(longer, c); ++retry) {
                            const int n = longer.sched_launches ? longer.sched_launches : 64;
                            const int m = n < kSchedRetryMaxLaunches / 4 ? 4 * n : kSchedRetryMaxLaunches;
                            if (m <= n) break;
                            longer.sched_launches = m;
                            rc = measure_cell_plain(ctx, &p->victims[v], &longer, &c);
                            if (rc) return rc;
                            fill_validity(c);
                        }
                    }
                }
        }
        *n_out = n;
        return IFR_OK;
    }
    // batched: one graph per (stressor, level) plus one for the solo runs
    const int n_graphs = 1 + p->n_stressors * (p->n_levels + 1);
    std::vector<cudaGraphExec_t> execs((size_t)n_graphs, nullptr);
    int slot = ifr_slot_alloc(ctx);
    if (slot < 0) return slot;
    rc = ifr_slot_prepare(ctx, slot);
    if (rc) return rc;
    ctx->slots[slot].watch = 1;
    std::vector<ifr_stressor_cfg> cfgs((size_t)n_graphs);
    struct Shape {
        int grid, block, planned, launches;
    };
    std::vector<Shape> shapes((size_t)n_graphs);
    std::vector<uint64_t> nodes((size_t)n_graphs, 0);
    for (int gi = 0; gi < n_graphs && !rc; ++gi) {
        if (gi == 0) {
            rc = capture_batch(ctx, p, nullptr, slot, &execs[0], &nodes[0]);
        } else {
            const int r = (gi - 1) / (p->n_levels + 1), l = (gi - 1) % (p->n_levels + 1);
            cfgs[gi] = level_cfg(p, r, l);
            rc = capture_batch(ctx, p, &cfgs[gi], slot, &execs[gi], &nodes[gi]);
            const Slot &s = ctx->slots[slot];
            shapes[gi] = Shape{s.grid, s.block, s.planned, s.launches};
        }
    }
    ctx->slots[slot].in_use = 1;
    std::vector<DevTiming> ht((size_t)p->n_victims);
    for (int rep = 0; rep < p->repeats && !rc; ++rep) {
        for (int gi = 0; gi < n_graphs && !rc; ++gi) {
            Slot &s = ctx->slots[slot];
            if (gi > 0) {
                s.cfg = cfgs[gi];
                s.grid = shapes[gi].grid;
                s.block = shapes[gi].block;
                s.planned = shapes[gi].planned;
                s.launches = shapes[gi].launches;
                s.in_use = 1;
                s.finished = 0;
            }
            cudaError_t e = cudaGraphLaunch(execs[gi], ctx->s_victim);
            ctx->kernel_launches += nodes[gi];
            if (e != cudaSuccess) {
                rc = ifr_cuda_fail(e, "cudaGraphLaunch", __FILE__, __LINE__);
                break;
            }
            e = cudaEventRecord(ctx->ev_b, ctx->s_victim);
            if (e != cudaSuccess) {
                rc = ifr_cuda_fail(e, "cudaEventRecord", __FILE__, __LINE__);
                break;
            }
            rc = wait_event_bounded(ctx->ev_b, 120000);
            if (rc) break;
            e = cudaMemcpy(ht.data(), ctx->d_timing, sizeof(DevTiming) * (size_t)p->n_victims, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                rc = ifr_cuda_fail(e, "cudaMemcpy timings", __FILE__, __LINE__);
                break;
            }
            ifr_stressor_result sres;
            memset(&sres, 0, sizeof sres);
            if (gi > 0) {
                rc = ifr_stressor_collect(ctx, slot);
                if (rc) break;
                sres = s.result;
                sres.elapsed_ms = 0.0;  // events are not recorded inside graphs
            }
            const int r = gi == 0 ? -1 : (gi - 1) / (p->n_levels + 1);
            const int l = gi == 0 ? 0 : (gi - 1) % (p->n_levels + 1);
            for (int v = 0; v < p->n_victims; ++v) {
                ifr_cell_result &c = cells[n++];
                memset(&c, 0, sizeof c);
                c.victim = v;
                c.stressor = r;
                c.level = l;
                c.repeat = rep;
                ifr_timing_to_host(ht[v], p->victims[v].repeats > 0 ? p->victims[v].repeats : 1, &c.timing);
                c.timing.event_ms = 0.0;
                if (gi > 0) {
                    c.stress = sres;
                    // the residency wait stamps its status into victim 0's slot only
                    if (v > 0 && ht[0].status != IFR_OK) c.timing.status = ht[0].status;
                }
                fill_validity(c);
            }
        }
    }
    ctx->slots[slot].in_use = 0;
    for (auto &e : execs)
        if (e) cudaGraphExecDestroy(e);
    *n_out = n;
    return rc;
}

int ifr_preload_sweep() {
    const void *fns[] = {(const void *)wait_started_kernel, (const void *)gate_kernel, (const void *)stamp_kernel};
    for (const void *f : fns) {
        int rc = ifr_preload(f);
        if (rc) return rc;
    }
    return IFR_OK;
}
