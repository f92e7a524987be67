// Slowdown-predictor MLP kernels: forward, backward, MSE gradient, Adam.
//
// The paper proposes (Sec. 5.1) a kernel-level interference estimator that
// predicts a kernel's slowdown from its metrics and resource sensitivity.  This
// library's estimator is a multilayer perceptron on the solo profiles of a victim
// and a co-runner; these are its inference and training kernels.
//
// Every GEMM of the network is  C[M][N] = sum_k A(m, k) B(k, n)  with bf16
// operands addressed through strides (so transposed operands need no copies) and
// fp32 accumulation on the tensor cores (warp-level mma.sync m16n8k16; the layers
// are 48..256 wide and a batch is 512 rows, so one launch is a few tiles and the
// cost is latency, not throughput).  Epilogues are fused:
//   forward hidden  Z = acc + b (fp32, kept for backward), H = bf16(GELU(Z))
//   forward output  Z = acc + b
//   backward dX     dZ_prev = acc * GELU'(Z_prev)  (fp32 for the bias gradient and
//                   bf16 for the next GEMMs)
//   backward dW     dW = acc (fp32)
// GELU is the exact erf form.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include "ifr_internal.cuh"

namespace {

constexpr int TM = 64, TN = 64, TK = 16, KPAD = 8;

enum Epi { EPI_FWD_HIDDEN = 0, EPI_FWD_OUT = 1, EPI_DX_GELU = 2, EPI_DW = 3, EPI_DX_PLAIN = 4 };

struct GemmArgs {
    const __nv_bfloat16 *A;
    int64_t a_rs, a_cs;  // A(m, k) = A[m * a_rs + k * a_cs]
    const __nv_bfloat16 *B;
    int64_t b_rs, b_cs;  // B(k, n) = B[k * b_rs + n * b_cs]
    int M, N, K;
    const float *bias;   // forward: [N]
    const float *Zin;    // backward dX: pre-activation of the previous layer [M][N]
    float *Zout;         // forward: pre-activation [M][N]
    __nv_bfloat16 *H;    // forward hidden: GELU output; backward dX: bf16 dZ_prev  [M][N]
    float *Out;          // backward dX: fp32 dZ_prev; dW: fp32 dW; dX plain: fp32 [M][N]
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One CTA = 64 x 64 output tile, 4 warps in a 2 x 2 grid of 32 x 32 warp tiles.
__global__ void __launch_bounds__(128) mlp_gemm_kernel(GemmArgs g, int epi) {
    __shared__ __align__(16) __nv_bfloat16 As[TM][TK + KPAD];  // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[TN][TK + KPAD];  // [n][k]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gq = lane >> 2, tq = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < g.K; k0 += TK) {
#pragma unroll
        for (int i = 0; i < (TM * TK) / 128; ++i) {
            const int idx = tid + i * 128, r = idx / TK, c = idx % TK;
            const int m = m0 + r, k = k0 + c, n = n0 + r;
            As[r][c] = (m < g.M && k < g.K) ? g.A[(int64_t)m * g.a_rs + (int64_t)k * g.a_cs] : zero;
            Bs[r][c] = (n < g.N && k < g.K) ? g.B[(int64_t)k * g.b_rs + (int64_t)n * g.b_cs] : zero;
        }
        __syncthreads();
        uint32_t af[2][4], bfr[4][2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int r = wm + mt * 16 + gq;
            af[mt][0] = *(const uint32_t *)&As[r][2 * tq];
            af[mt][1] = *(const uint32_t *)&As[r + 8][2 * tq];
            af[mt][2] = *(const uint32_t *)&As[r][2 * tq + 8];
            af[mt][3] = *(const uint32_t *)&As[r + 8][2 * tq + 8];
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int r = wn + nt * 8 + gq;
            bfr[nt][0] = *(const uint32_t *)&Bs[r][2 * tq];
            bfr[nt][1] = *(const uint32_t *)&Bs[r][2 * tq + 8];
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) mma16816(acc[mt][nt], af[mt], bfr[nt]);
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm + mt * 16 + gq + (r >= 2 ? 8 : 0);
                const int n = n0 + wn + nt * 8 + 2 * tq + (r & 1);
                if (m >= g.M || n >= g.N) continue;
                const int64_t o = (int64_t)m * g.N + n;
                const float v = acc[mt][nt][r];
                switch (epi) {
                    case EPI_FWD_HIDDEN: {
                        const float z = v + g.bias[n];
                        g.Zout[o] = z;
                        g.H[o] = __float2bfloat16_rn(gelu(z));
                        break;
                    }
                    case EPI_FWD_OUT: g.Zout[o] = v + g.bias[n]; break;
                    case EPI_DX_GELU: {
                        const float d = v * gelu_grad(g.Zin[o]);
                        g.Out[o] = d;
                        g.H[o] = __float2bfloat16_rn(d);
                        break;
                    }
                    default: g.Out[o] = v; break;
                }
            }
}

__global__ void copy_bf16_kernel(const float *__restrict__ x, float *__restrict__ y, __nv_bfloat16 *__restrict__ yh,
                                 int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        y[i] = x[i];
        yh[i] = __float2bfloat16_rn(x[i]);
    }
}

// db[n] = sum_m dZ[m][n]   (one thread per column, fixed summation order)
__global__ void colsum_kernel(const float *__restrict__ dZ, int M, int N, float *__restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += dZ[(int64_t)m * N + n];
    db[n] = s;
}

// loss = mean((yhat - t)^2), dY = 2 (yhat - t) / n (fp32 and bf16); one block.
__global__ void mse_grad_kernel(const float *__restrict__ yhat, const float *__restrict__ t, int n,
                                float *__restrict__ dY, __nv_bfloat16 *__restrict__ dYh, float *__restrict__ loss) {
    __shared__ float red[32];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = yhat[i] - t[i];
        const float gq = 2.f * d / (float)n;
        dY[i] = gq;
        if (dYh) dYh[i] = __float2bfloat16_rn(gq);
        s += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) tot += red[w];
        if (loss) *loss = tot / (float)n;
    }
}

// Adam (Kingma & Ba): m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
// w <- w - lr * mhat / (sqrt(vhat) + eps); optional bf16 copy of w.
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ wh, int64_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wh) wh[i] = __float2bfloat16_rn(wi);
    }
}

int launch_gemm(const GemmArgs &g, int epi, cudaStream_t s) {
    dim3 grid((unsigned)((g.N + TN - 1) / TN), (unsigned)((g.M + TM - 1) / TM));
    mlp_gemm_kernel<<<grid, 128, 0, s>>>(g, epi);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IFR_OK : ifr_cuda_fail(e, "mlp_gemm_kernel", __FILE__, __LINE__);
}

int check_mlp(const ifr_mlp *p) {
    if (!p || p->n_layers <= 0 || p->n_layers > IFR_MLP_MAX_LAYERS || p->batch <= 0) return IFR_ERR_ARG;
    for (int l = 0; l <= p->n_layers; ++l)
        if (p->dims[l] <= 0 || p->dims[l] > 65536) return IFR_ERR_ARG;
    if (p->dims[p->n_layers] != 1) return IFR_ERR_ARG;
    for (int l = 0; l < p->n_layers; ++l)
        if (!p->W[l] || !p->b[l] || !p->H[l] || !p->Z[l]) return IFR_ERR_ARG;
    return IFR_OK;
}

}  // namespace

extern "C" int ifr_mlp_forward(ifr_ctx *ctx, const ifr_mlp *p, void *stream) {
    if (!ctx) return IFR_ERR_ARG;
    int rc = check_mlp(p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = p->n_layers, B = p->batch;
    for (int l = 0; l < L; ++l) {
        GemmArgs g;
        memset(&g, 0, sizeof g);
        const int K = p->dims[l], N = p->dims[l + 1];
        g.A = (const __nv_bfloat16 *)p->H[l];
        g.a_rs = K;
        g.a_cs = 1;
        g.B = (const __nv_bfloat16 *)p->W[l];  // B(k, n) = W[n][k]
        g.b_rs = 1;
        g.b_cs = K;
        g.M = B;
        g.N = N;
        g.K = K;
        g.bias = p->b[l];
        g.Zout = p->Z[l];
        const bool hidden = l < L - 1;
        if (hidden) {
            if (!p->H[l + 1]) return IFR_ERR_ARG;
            g.H = (__nv_bfloat16 *)p->H[l + 1];
        }
        rc = launch_gemm(g, hidden ? EPI_FWD_HIDDEN : EPI_FWD_OUT, s);
        if (rc) return rc;
        ctx->kernel_launches += 1;
    }
    return IFR_OK;
}

extern "C" int ifr_mlp_backward(ifr_ctx *ctx, const ifr_mlp *p, const float *dY, void *stream) {
    if (!ctx || !dY) return IFR_ERR_ARG;
    int rc = check_mlp(p);
    if (rc) return rc;
    const int L = p->n_layers, B = p->batch;
    for (int l = 0; l < L; ++l)
        if (!p->dW[l] || !p->db[l] || !p->dZ[l] || !p->dZh[l]) return IFR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // the output layer's dZ is dY itself (fp32 and bf16 copies)
    copy_bf16_kernel<<<(B + 255) / 256, 256, 0, s>>>(dY, p->dZ[L - 1], (__nv_bfloat16 *)p->dZh[L - 1], B);
    IFR_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    for (int l = L - 1; l >= 0; --l) {
        const int K = p->dims[l], N = p->dims[l + 1];
        // dW[n][k] = sum_m dZ(m, n) H(m, k)
        GemmArgs g;
        memset(&g, 0, sizeof g);
        g.A = (const __nv_bfloat16 *)p->dZh[l];  // A(n, m) = dZ[m][n]
        g.a_rs = 1;
        g.a_cs = N;
        g.B = (const __nv_bfloat16 *)p->H[l];  // B(m, k) = H[m][k]
        g.b_rs = K;
        g.b_cs = 1;
        g.M = N;
        g.N = K;
        g.K = B;
        g.Out = p->dW[l];
        rc = launch_gemm(g, EPI_DW, s);
        if (rc) return rc;
        colsum_kernel<<<(N + 127) / 128, 128, 0, s>>>(p->dZ[l], B, N, p->db[l]);
        IFR_CUDA(cudaGetLastError());
        ctx->kernel_launches += 2;
        if (l == 0 && !p->dX) break;
        // dH(m, k) = sum_n dZ(m, n) W[n][k]; below the first layer: times GELU'(Z_prev)
        GemmArgs h;
        memset(&h, 0, sizeof h);
        h.A = (const __nv_bfloat16 *)p->dZh[l];  // A(m, n) = dZ[m][n]
        h.a_rs = N;
        h.a_cs = 1;
        h.B = (const __nv_bfloat16 *)p->W[l];  // B(n, k) = W[n][k]
        h.b_rs = K;
        h.b_cs = 1;
        h.M = B;
        h.N = K;
        h.K = N;
        if (l > 0) {
            h.Zin = p->Z[l - 1];
            h.Out = p->dZ[l - 1];
            h.H = (__nv_bfloat16 *)p->dZh[l - 1];
            rc = launch_gemm(h, EPI_DX_GELU, s);
        } else {
            h.Out = p->dX;
            rc = launch_gemm(h, EPI_DX_PLAIN, s);
        }
        if (rc) return rc;
        ctx->kernel_launches += 1;
    }
    return IFR_OK;
}

extern "C" int ifr_mse_grad(ifr_ctx *ctx, const float *yhat, const float *target, int n, float *dY, float *loss,
                            void *stream) {
    if (!ctx || !yhat || !target || !dY || n <= 0) return IFR_ERR_ARG;
    mse_grad_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(yhat, target, n, dY, nullptr, loss);
    IFR_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    return IFR_OK;
}

extern "C" int ifr_adam_step(ifr_ctx *ctx, float *w, const float *g, float *m, float *v, void *w_bf16, int64_t n,
                             float lr, float beta1, float beta2, float eps, int step, void *stream) {
    if (!ctx || !w || !g || !m || !v || n <= 0 || step <= 0) return IFR_ERR_ARG;
    const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
    const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
    int grid = (int)((n + 255) / 256);
    if (grid > ctx->info.num_sms * 8) grid = ctx->info.num_sms * 8;
    adam_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(w, g, m, v, (__nv_bfloat16 *)w_bf16, n, lr, beta1, beta2, eps,
                                                        c1, c2);
    IFR_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    return IFR_OK;
}

int ifr_preload_mlp() {
    const void *fns[] = {(const void *)mlp_gemm_kernel, (const void *)copy_bf16_kernel, (const void *)colsum_kernel,
                         (const void *)mse_grad_kernel, (const void *)adam_kernel};
    for (const void *f : fns) {
        int rc = ifr_preload(f);
        if (rc) return rc;
    }
    return IFR_OK;
}
