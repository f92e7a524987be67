// BF16 tensor-pipe stressor (tcgen05) — placeholder until the tcgen05 path lands.
#include "ifr_internal.cuh"

int ifr_tensor_stressor_launch(const StressParams &, DevStress *, int, int, cudaStream_t) {
    return IFR_ERR_UNSUPPORTED;
}
