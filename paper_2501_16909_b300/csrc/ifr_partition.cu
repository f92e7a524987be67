// SM partitions with CUDA green contexts (Sec. 4.1: inter-SM colocation runs each
// workload in its own green context, a disjoint SM set with its own stream).  The
// driver entry points are looked up at run time, so the library needs no link
// dependency on the driver library.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "ifr_internal.cuh"

namespace {

struct GreenApi {
    PFN_cuDeviceGet_v2000 device_get = nullptr;
    PFN_cuDeviceGetDevResource_v12040 get_resource = nullptr;
    PFN_cuDevSmResourceSplitByCount_v12040 split = nullptr;
    PFN_cuDevResourceGenerateDesc_v12040 gen_desc = nullptr;
    PFN_cuGreenCtxCreate_v12040 create = nullptr;
    PFN_cuGreenCtxDestroy_v12040 destroy = nullptr;
    PFN_cuGreenCtxStreamCreate_v12050 stream_create = nullptr;
    PFN_cuStreamDestroy_v4000 stream_destroy = nullptr;
    bool ok = false;
};

template <typename F>
bool entry(const char *name, int version, F *out) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    *out = (F)p;
    return true;
}

const GreenApi &api() {
    static GreenApi a;
    static bool tried = false;
    if (!tried) {
        tried = true;
        a.ok = entry("cuDeviceGet", 2000, &a.device_get) && entry("cuDeviceGetDevResource", 12040, &a.get_resource) &&
               entry("cuDevSmResourceSplitByCount", 12040, &a.split) &&
               entry("cuDevResourceGenerateDesc", 12040, &a.gen_desc) && entry("cuGreenCtxCreate", 12040, &a.create) &&
               entry("cuGreenCtxDestroy", 12040, &a.destroy) &&
               entry("cuGreenCtxStreamCreate", 12050, &a.stream_create) &&
               entry("cuStreamDestroy", 4000, &a.stream_destroy);
    }
    return a;
}

}  // namespace

extern "C" int ifr_partition_release(ifr_ctx *ctx) {
    if (!ctx) return IFR_ERR_ARG;
    if (!ctx->part_active) return IFR_OK;
    IFR_CUDA(cudaDeviceSynchronize());
    const GreenApi &a = api();
    a.stream_destroy((CUstream)ctx->s_victim);
    a.stream_destroy((CUstream)ctx->s_stress);
    a.destroy((CUgreenCtx)ctx->green_v);
    a.destroy((CUgreenCtx)ctx->green_s);
    ctx->s_victim = ctx->own_victim;
    ctx->s_stress = ctx->own_stress;
    ctx->green_v = ctx->green_s = nullptr;
    ctx->part_active = 0;
    ctx->part_sms_v = ctx->part_sms_s = 0;
    return IFR_OK;
}

extern "C" int ifr_partition(ifr_ctx *ctx, int victim_sms, int flags, ifr_partition_info *out) {
    if (!ctx || !out || ctx->part_active || victim_sms < 1 || victim_sms >= ctx->info.num_sms || (flags & ~1))
        return IFR_ERR_ARG;
    const GreenApi &a = api();
    if (!a.ok) return IFR_ERR_UNSUPPORTED;
    memset(out, 0, sizeof *out);
    IFR_CUDA(cudaDeviceSynchronize());
    CUdevice dev;
    if (a.device_get(&dev, ctx->device) != CUDA_SUCCESS) return IFR_ERR_UNSUPPORTED;
    CUdevResource all, group, rest;
    memset(&rest, 0, sizeof rest);
    if (a.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) return IFR_ERR_UNSUPPORTED;
    unsigned nb = 1;
    const unsigned use = (flags & 1) ? CU_DEV_SM_RESOURCE_SPLIT_IGNORE_SM_COSCHEDULING : 0u;
    if (a.split(&group, &nb, &all, &rest, use, (unsigned)victim_sms) != CUDA_SUCCESS || nb != 1 ||
        rest.sm.smCount == 0)
        return IFR_ERR_UNSUPPORTED;
    CUdevResourceDesc dv, ds;
    if (a.gen_desc(&dv, &group, 1) != CUDA_SUCCESS || a.gen_desc(&ds, &rest, 1) != CUDA_SUCCESS)
        return IFR_ERR_UNSUPPORTED;
    CUgreenCtx gv = nullptr, gs = nullptr;
    CUstream sv = nullptr, ss = nullptr;
    int rc = IFR_ERR_UNSUPPORTED;
    if (a.create(&gv, dv, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
        a.create(&gs, ds, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
        a.stream_create(&sv, gv, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS &&
        a.stream_create(&ss, gs, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS)
        rc = IFR_OK;
    if (rc != IFR_OK) {
        if (sv) a.stream_destroy(sv);
        if (ss) a.stream_destroy(ss);
        if (gv) a.destroy(gv);
        if (gs) a.destroy(gs);
        return rc;
    }
    ctx->own_victim = ctx->s_victim;
    ctx->own_stress = ctx->s_stress;
    ctx->s_victim = (cudaStream_t)sv;
    ctx->s_stress = (cudaStream_t)ss;
    ctx->green_v = gv;
    ctx->green_s = gs;
    ctx->part_sms_v = (int)group.sm.smCount;
    ctx->part_sms_s = (int)rest.sm.smCount;
    ctx->part_active = 1;
    out->victim_sms = ctx->part_sms_v;
    out->stressor_sms = ctx->part_sms_s;
    return IFR_OK;
}
