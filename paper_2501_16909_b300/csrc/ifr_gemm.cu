// BF16 GEMM victim (tcgen05) — placeholder until the tcgen05 path lands.
#include "ifr_internal.cuh"

int ifr_gemm_enqueue(ifr_ctx *, const ifr_victim_cfg *, cudaStream_t, DevTiming *) { return IFR_ERR_UNSUPPORTED; }
