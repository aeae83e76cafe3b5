// mlp.cu -- the learned surrogate of <<v>>: an ensemble of multilayer
// perceptrons trained and evaluated by the library's own kernels.
//
// Layer l computes z = h W_l^T + b_l; hidden layers apply SiLU, z / (1 +
// e^-z).  Loss: mean over the batch of (out - y)^2.  Backward: dW_l =
// dZ_l^T h_l, db_l = column sums of dZ_l, dH_{l-1} = dZ_l W_l, dZ_{l-1} =
// dH_{l-1} * SiLU'(z_{l-1}).  Adam (Kingma & Ba, Algorithm 1) on FP32 master
// weights.  Every GEMM reads BF16 operands (weights and activations rounded
// from FP32) and accumulates in FP32; pre-activations are kept in FP32.
//
// Inference (sde_mlp_forward) of width-256 networks with at least two hidden
// layers runs the fused tensor-core kernel of mlp_tc.cuh: the square hidden
// layers as tcgen05 MMAs (M = 128 points, N = 256, K = 256) with the bias,
// SiLU and the output layer in their epilogues.  The training path (forward
// with stored pre-activations, backward, Adam) uses one tiled CUDA-core kernel
// with 64 x 64 output tiles for all three GEMM shapes (forward, weight
// gradient, input gradient) through layout flags, with the bias / activation /
// derivative fused into its epilogue.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "mlp_tc.cuh"
#include "philox.cuh"
#include "tma_map.h"

using sde::cuda_fail;
using sde::set_error;

namespace sde {
namespace {

constexpr uint32_t kTagInit = 6u;  // Philox stream tag of the initial weights

enum Epi { EPI_FWD_HIDDEN = 0, EPI_FWD_OUT = 1, EPI_STORE = 2, EPI_DSILU = 3 };

__device__ __forceinline__ float ld(const float *p) { return *p; }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

struct EpiArgs {
  const float *bias;      // FWD_*: bias[n]
  float *zout;            // FWD_HIDDEN: pre-activation [M][N]; FWD_OUT / STORE: output [M][N]
  __nv_bfloat16 *hout;    // FWD_HIDDEN: SiLU(z) [M][N]; DSILU: dZ [M][N]
  const float *zin;       // DSILU: pre-activation [M][N]
};

// C[m][n] = sum_k A(m, k) B(n, k);
// A(m, k) = A_T ? A[k * M + m] : A[m * K + k];  B(n, k) = B_T ? B[k * N + n] : B[n * K + k].
template <typename TA, typename TB, bool A_T, bool B_T, int EPI>
__global__ void __launch_bounds__(256) mlp_gemm_kernel(const TA *__restrict__ A, const TB *__restrict__ Bm,
                                                       int M, int N, int K, EpiArgs e) {
  constexpr int TM = 64, TN = 64, TK = 16;
  __shared__ float As[TK][TM + 4];
  __shared__ float Bs[TK][TN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int el = tid * 4 + q;  // 1024 elements of each tile
      int m, k;
      if (A_T) {
        k = el / TM;
        m = el % TM;
      } else {
        m = el / TK;
        k = el % TK;
      }
      const int gm = m0 + m, gk = k0 + k;
      float a = 0.0f;
      if (gm < M && gk < K) a = A_T ? ld(A + (size_t)gk * M + gm) : ld(A + (size_t)gm * K + gk);
      As[k][m] = a;
      int n, kb;
      if (B_T) {
        kb = el / TN;
        n = el % TN;
      } else {
        n = el / TK;
        kb = el % TK;
      }
      const int gn = n0 + n, gkb = k0 + kb;
      float b = 0.0f;
      if (gn < N && gkb < K) b = B_T ? ld(Bm + (size_t)gkb * N + gn) : ld(Bm + (size_t)gn * K + gkb);
      Bs[kb][n] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        b[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      const size_t o = (size_t)m * N + n;
      if (EPI == EPI_FWD_HIDDEN) {
        const float z = acc[i][j] + e.bias[n];
        e.zout[o] = z;
        e.hout[o] = __float2bfloat16_rn(z * sigmoidf_(z));
      } else if (EPI == EPI_FWD_OUT) {
        e.zout[o] = acc[i][j] + e.bias[n];
      } else if (EPI == EPI_STORE) {
        e.zout[o] = acc[i][j];
      } else {
        const float z = e.zin[o];
        const float s = sigmoidf_(z);
        e.hout[o] = __float2bfloat16_rn(acc[i][j] * (s * (1.0f + z * (1.0f - s))));
      }
    }
  }
}

__global__ void to_bf16_kernel(const float *src, __nv_bfloat16 *dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

// Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights and biases.
__global__ void init_kernel(float *params, const int64_t *off, const int *fin, int L, int64_t P, int member,
                            uint64_t seed) {
  const uint2 key = seed_to_key(seed);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
    int l = 0;
    while (l + 1 < L && i >= off[l + 1]) ++l;
    const float bound = rsqrtf((float)fin[l]);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)member, kTagInit), key);
    params[(int64_t)member * P + i] = (2.0f * uniform24(r.x) - 1.0f) * bound;
  }
}

// out = 2/B (y_pred - y), loss = mean (y_pred - y)^2 (one block, fixed order).
__global__ void loss_kernel(const float *pred, const float *y, int64_t B, float *g, float *loss) {
  __shared__ float red[32];
  float s = 0.0f;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
    const float d = pred[b] - y[b];
    g[b] = 2.0f * d / (float)B;
    s += d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0 && loss) *loss = s / (float)B;
  }
}

// db[n] = sum_b dZ[b][n]: one block per column, fixed order.
template <typename T>
__global__ void colsum_kernel(const T *dz, int64_t B, int N, float *db) {
  __shared__ float red[32];
  const int n = blockIdx.x;
  float s = 0.0f;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) s += ld(dz + b * N + n);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) db[n] = s;
  }
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr_t, float b1,
                            float b2, float eps_t) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr_t * mi / (sqrtf(vi) + eps_t);
  }
}

__global__ void features_kernel(const sde_jj_point *pts, int64_t n, float *X, const float *lo_hi) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const sde_jj_point p = pts[i];
    const double raw[5] = {p.a, p.omega, p.f, p.gamma, log10(p.D)};
#pragma unroll
    for (int k = 0; k < 5; ++k)
      X[i * 5 + k] = (float)(2.0 * (raw[k] - (double)lo_hi[k]) / ((double)lo_hi[5 + k] - (double)lo_hi[k]) - 1.0);
  }
}

// Mean and standard deviation over the members' outputs (rows `stride` apart).
__global__ void ensemble_stats_kernel(const float *out, int members, int64_t stride, int64_t B, float *mean,
                                      float *spread) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B; b += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < members; ++q) s += out[(int64_t)q * stride + b];
    const double mu = s / members;
    double m2 = 0.0;
    for (int q = 0; q < members; ++q) {
      const double d = out[(int64_t)q * stride + b] - mu;
      m2 += d * d;
    }
    mean[b] = (float)mu;
    if (spread) spread[b] = members > 1 ? (float)sqrt(m2 / (members - 1)) : 0.0f;
  }
}

int grid1(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

// BF16 copies of the square hidden layers' weights for the tensor-core
// forward: whh[member][l][n][k] = W_{l+1}[n][k] of that member.
struct SquareOffsets {
  int64_t w[mlptc::MAX_HH];
};

__global__ void square_weights_kernel(const float *params, int64_t P, int members, int n_hh, SquareOffsets off,
                                      __nv_bfloat16 *whh) {
  constexpr int64_t HH = (int64_t)mlptc::H * mlptc::H;
  const int64_t n = (int64_t)members * n_hh * HH;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ml = i / HH;
    const int member = (int)(ml / n_hh), l = (int)(ml % n_hh);
    whh[i] = __float2bfloat16_rn(params[(int64_t)member * P + off.w[l] + (i - ml * HH)]);
  }
}

}  // namespace
}  // namespace sde

struct sde_mlp {
  sde_mlp_config cfg{};
  int L = 0;                    // linear layers
  std::vector<int> fin, fout;   // per layer
  std::vector<int64_t> woff, boff;
  int64_t P = 0;                // parameters per member
  float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;  // [members][P]
  __nv_bfloat16 *wbf = nullptr;                                         // [P]
  std::vector<__nv_bfloat16 *> h;  // L entries: layer inputs (bf16), h[0] = X
  std::vector<float *> z;          // L - 1 hidden pre-activations
  __nv_bfloat16 *dz[2] = {nullptr, nullptr};
  float *out = nullptr;            // [members][B]
  float *gout = nullptr;           // [B] output-layer gradient
  float *lo_hi = nullptr;          // [10]
  int64_t *off_dev = nullptr;
  int *fin_dev = nullptr;
  int64_t step = 0;
  // tensor-core forward (width 256, at least two hidden layers)
  bool tc = false;                 // the shape has the tensor-core path
  bool use_tc = true;              // sde_mlp_use_tensor_cores
  __nv_bfloat16 *whh = nullptr;    // [members][n_hidden - 1][256][256]
  CUtensorMap map_whh;
  uint32_t *err = nullptr;         // latched kErrTimeout of the tensor-core kernel
};

namespace {

using namespace sde;

template <typename TA, typename TB, bool A_T, bool B_T, int EPI>
cudaError_t gemm(const TA *A, const TB *B, int M, int N, int K, EpiArgs e, cudaStream_t s) {
  dim3 grid((M + 63) / 64, (N + 63) / 64);
  mlp_gemm_kernel<TA, TB, A_T, B_T, EPI><<<grid, 256, 0, s>>>(A, B, M, N, K, e);
  return cudaGetLastError();
}

// Forward pass of one member over X (FP32 [B][n_in]); output -> out_row[B].
sde_status mlp_forward_member(sde_mlp *q, int member, const float *X, int64_t B, float *out_row, cudaStream_t s) {
  SDE_CUDA_TRY(cudaGetLastError());
  to_bf16_kernel<<<grid1(q->P), 256, 0, s>>>(q->params + (int64_t)member * q->P, q->wbf, q->P);
  to_bf16_kernel<<<grid1(B * q->cfg.n_in), 256, 0, s>>>(X, q->h[0], B * q->cfg.n_in);
  SDE_CUDA_TRY(cudaGetLastError());
  const float *pm = q->params + (int64_t)member * q->P;
  for (int l = 0; l < q->L; ++l) {
    EpiArgs e{};
    e.bias = pm + q->boff[l];
    if (l < q->L - 1) {
      e.zout = q->z[l];
      e.hout = q->h[l + 1];
      SDE_CUDA_TRY((gemm<__nv_bfloat16, __nv_bfloat16, false, false, EPI_FWD_HIDDEN>(
          q->h[l], q->wbf + q->woff[l], (int)B, q->fout[l], q->fin[l], e, s)));
    } else {
      e.zout = out_row;
      SDE_CUDA_TRY((gemm<__nv_bfloat16, __nv_bfloat16, false, false, EPI_FWD_OUT>(
          q->h[l], q->wbf + q->woff[l], (int)B, q->fout[l], q->fin[l], e, s)));
    }
  }
  return SDE_OK;
}

// Gradient of the MSE of one member into grad_out[P]; loss -> loss_out.
sde_status mlp_grad_member(sde_mlp *q, int member, const float *X, const float *y, int64_t B, float *grad_out,
                           float *loss_out, cudaStream_t s) {
  float *pred = q->out + (int64_t)member * q->cfg.max_batch;
  sde_status st = mlp_forward_member(q, member, X, B, pred, s);
  if (st != SDE_OK) return st;
  loss_kernel<<<1, 1024, 0, s>>>(pred, y, B, q->gout, loss_out);
  SDE_CUDA_TRY(cudaGetLastError());
  int cur = 0;
  for (int l = q->L - 1; l >= 0; --l) {
    EpiArgs e{};
    // weight gradient dW_l = dZ_l^T h_l  ([fout][fin], K = batch)
    e.zout = grad_out + q->woff[l];
    if (l == q->L - 1) {
      SDE_CUDA_TRY((gemm<float, __nv_bfloat16, true, true, EPI_STORE>(q->gout, q->h[l], q->fout[l], q->fin[l],
                                                                       (int)B, e, s)));
      colsum_kernel<float><<<q->fout[l], 256, 0, s>>>(q->gout, B, q->fout[l], grad_out + q->boff[l]);
    } else {
      SDE_CUDA_TRY((gemm<__nv_bfloat16, __nv_bfloat16, true, true, EPI_STORE>(q->dz[cur], q->h[l], q->fout[l],
                                                                               q->fin[l], (int)B, e, s)));
      colsum_kernel<__nv_bfloat16><<<q->fout[l], 256, 0, s>>>(q->dz[cur], B, q->fout[l], grad_out + q->boff[l]);
    }
    SDE_CUDA_TRY(cudaGetLastError());
    if (l > 0) {
      // dZ_{l-1} = (dZ_l W_l) * SiLU'(z_{l-1})   ([B][fin])
      EpiArgs d{};
      d.zin = q->z[l - 1];
      d.hout = q->dz[cur ^ 1];
      if (l == q->L - 1)
        SDE_CUDA_TRY((gemm<float, __nv_bfloat16, false, true, EPI_DSILU>(q->gout, q->wbf + q->woff[l], (int)B,
                                                                         q->fin[l], q->fout[l], d, s)));
      else
        SDE_CUDA_TRY((gemm<__nv_bfloat16, __nv_bfloat16, false, true, EPI_DSILU>(
            q->dz[cur], q->wbf + q->woff[l], (int)B, q->fin[l], q->fout[l], d, s)));
      cur ^= 1;
    }
  }
  return SDE_OK;
}

void mlp_free(sde_mlp *q) {
  if (!q) return;
  cudaDeviceSynchronize();
  cudaFree(q->params);
  cudaFree(q->m);
  cudaFree(q->v);
  cudaFree(q->grad);
  cudaFree(q->wbf);
  for (auto p : q->h) cudaFree(p);
  for (auto p : q->z) cudaFree(p);
  cudaFree(q->dz[0]);
  cudaFree(q->dz[1]);
  cudaFree(q->out);
  cudaFree(q->gout);
  cudaFree(q->lo_hi);
  cudaFree(q->off_dev);
  cudaFree(q->fin_dev);
  cudaFree(q->whh);
  cudaFree(q->err);
  delete q;
}

}  // namespace

using namespace sde;

extern "C" {

sde_status sde_mlp_create(const sde_mlp_config *cfg, sde_mlp **out) {
  clear_error();
  SDE_CHECK_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  SDE_CHECK_ARG(cfg != nullptr, "cfg is NULL");
  SDE_CHECK_ARG(cfg->n_in >= 1 && cfg->n_in <= 8, "n_in must be in [1, 8]");
  SDE_CHECK_ARG(cfg->hidden >= 64 && cfg->hidden <= 1024 && cfg->hidden % 64 == 0,
                "hidden must be a multiple of 64 in [64, 1024]");
  SDE_CHECK_ARG(cfg->n_hidden >= 1 && cfg->n_hidden <= 8, "n_hidden must be in [1, 8]");
  SDE_CHECK_ARG(cfg->n_members >= 1 && cfg->n_members <= 16, "n_members must be in [1, 16]");
  SDE_CHECK_ARG(cfg->max_batch >= 1 && cfg->max_batch <= (1ll << 24), "max_batch must be in [1, 2^24]");
  SDE_CHECK_ARG(cfg->lr > 0.0f && cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f && cfg->beta2 >= 0.0f &&
                    cfg->beta2 < 1.0f && cfg->eps > 0.0f,
                "Adam hyper-parameters out of range");
  for (int k = 0; k < 5; ++k) SDE_CHECK_ARG(cfg->hi[k] > cfg->lo[k], "feature box needs hi > lo");
  sde_mlp *q = new (std::nothrow) sde_mlp();
  if (!q) {
    set_error("host allocation failed");
    return SDE_ERR_NO_MEMORY;
  }
  q->cfg = *cfg;
  q->L = cfg->n_hidden + 1;
  int64_t off = 0;
  for (int l = 0; l < q->L; ++l) {
    const int fi = l == 0 ? cfg->n_in : cfg->hidden;
    const int fo = l == q->L - 1 ? 1 : cfg->hidden;
    q->fin.push_back(fi);
    q->fout.push_back(fo);
    q->woff.push_back(off);
    off += (int64_t)fi * fo;
    q->boff.push_back(off);
    off += fo;
  }
  q->P = off;
  const int64_t M = cfg->n_members, B = cfg->max_batch, H = cfg->hidden;
  sde_status st = SDE_OK;
  auto alloc = [&](void **p, size_t bytes) {
    if (st != SDE_OK) return;
    cudaError_t e = device_alloc(p, bytes ? bytes : 1);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc");
  };
  alloc((void **)&q->params, sizeof(float) * M * q->P);
  alloc((void **)&q->m, sizeof(float) * M * q->P);
  alloc((void **)&q->v, sizeof(float) * M * q->P);
  alloc((void **)&q->grad, sizeof(float) * M * q->P);
  alloc((void **)&q->wbf, sizeof(__nv_bfloat16) * q->P);
  q->h.assign(q->L, nullptr);
  q->z.assign(q->L - 1, nullptr);
  alloc((void **)&q->h[0], sizeof(__nv_bfloat16) * B * cfg->n_in);
  for (int l = 1; l < q->L; ++l) alloc((void **)&q->h[l], sizeof(__nv_bfloat16) * B * H);
  for (int l = 0; l < q->L - 1; ++l) alloc((void **)&q->z[l], sizeof(float) * B * H);
  alloc((void **)&q->dz[0], sizeof(__nv_bfloat16) * B * H);
  alloc((void **)&q->dz[1], sizeof(__nv_bfloat16) * B * H);
  alloc((void **)&q->out, sizeof(float) * M * B);
  alloc((void **)&q->gout, sizeof(float) * B);
  alloc((void **)&q->lo_hi, sizeof(float) * 10);
  alloc((void **)&q->off_dev, sizeof(int64_t) * (q->L + 1));
  alloc((void **)&q->fin_dev, sizeof(int) * q->L);
  alloc((void **)&q->err, sizeof(uint32_t));
  q->tc = cfg->hidden == mlptc::H && cfg->n_hidden >= 2 && cfg->n_hidden - 1 <= mlptc::MAX_HH &&
          cfg->n_in <= mlptc::MAX_IN;
  if (q->tc) alloc((void **)&q->whh, sizeof(__nv_bfloat16) * M * (cfg->n_hidden - 1) * H * H);
  alloc_injection_disarm();
  if (st == SDE_OK && q->tc) {
    st = make_map_bf16(&q->map_whh, q->whh, M * (cfg->n_hidden - 1) * H, H, mlptc::H);
    if (st == SDE_OK) {
      const cudaError_t e = cudaFuncSetAttribute(mlptc::mlp_fwd_tc_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, mlptc::SMEM_BYTES);
      if (e != cudaSuccess) st = cuda_fail(e, "cudaFuncSetAttribute(mlp_fwd_tc_kernel)");
    }
  }
  if (st == SDE_OK) {
    float lh[10];
    for (int k = 0; k < 5; ++k) {
      lh[k] = cfg->lo[k];
      lh[5 + k] = cfg->hi[k];
    }
    std::vector<int64_t> offs(q->woff.begin(), q->woff.end());
    offs.push_back(q->P);
    cudaError_t e = cudaMemcpy(q->lo_hi, lh, sizeof lh, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q->off_dev, offs.data(), sizeof(int64_t) * offs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q->fin_dev, q->fin.data(), sizeof(int) * q->L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(q->m, 0, sizeof(float) * M * q->P);
    if (e == cudaSuccess) e = cudaMemset(q->err, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(q->v, 0, sizeof(float) * M * q->P);
    for (int mm = 0; mm < M && e == cudaSuccess; ++mm) {
      init_kernel<<<grid1(q->P), 256>>>(q->params, q->off_dev, q->fin_dev, q->L, q->P, mm, cfg->seed);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_fail(e, "sde_mlp_create");
  }
  if (st != SDE_OK) {
    std::string msg = sde_last_error();
    mlp_free(q);
    set_error(msg);
    return st;
  }
  *out = q;
  return SDE_OK;
}

void sde_mlp_destroy(sde_mlp *q) { mlp_free(q); }

int64_t sde_mlp_num_params(const sde_mlp *q) { return q ? q->P : -1; }

sde_status sde_mlp_set_params(sde_mlp *q, int32_t member, const float *p, void *stream) {
  clear_error();
  SDE_CHECK_ARG(q && p, "mlp and params must be non-NULL");
  SDE_CHECK_ARG(member >= 0 && member < q->cfg.n_members, "member out of range");
  SDE_CUDA_TRY(cudaMemcpyAsync(q->params + (int64_t)member * q->P, p, sizeof(float) * q->P,
                               cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return SDE_OK;
}

sde_status sde_mlp_get_params(sde_mlp *q, int32_t member, float *p, void *stream) {
  clear_error();
  SDE_CHECK_ARG(q && p, "mlp and params must be non-NULL");
  SDE_CHECK_ARG(member >= 0 && member < q->cfg.n_members, "member out of range");
  SDE_CUDA_TRY(cudaMemcpyAsync(p, q->params + (int64_t)member * q->P, sizeof(float) * q->P,
                               cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return SDE_OK;
}

sde_status sde_mlp_features(sde_mlp *q, const sde_jj_point *pts, int64_t n, float *X, void *stream) {
  clear_error();
  SDE_CHECK_ARG(q != nullptr && n >= 0, "mlp is NULL or n < 0");
  SDE_CHECK_ARG(q->cfg.n_in == 5, "the parameter features need n_in == 5");
  if (n == 0) return SDE_OK;
  SDE_CHECK_ARG(pts && X, "points and X must be non-NULL");
  features_kernel<<<grid1(n), 256, 0, (cudaStream_t)stream>>>(pts, n, X, q->lo_hi);
  SDE_CUDA_TRY(cudaGetLastError());
  return SDE_OK;
}

sde_status sde_mlp_forward(sde_mlp *q, const float *X, int64_t B, float *mean, float *spread, void *stream) {
  clear_error();
  SDE_CHECK_ARG(q != nullptr, "mlp is NULL");
  SDE_CHECK_ARG(B >= 0 && B <= q->cfg.max_batch, "batch exceeds max_batch");
  if (B == 0) return SDE_OK;
  SDE_CHECK_ARG(X && mean, "X and mean must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (q->tc && q->use_tc) {
    const int n_hh = q->cfg.n_hidden - 1;
    SquareOffsets so{};
    mlptc::Args a{};
    for (int l = 0; l < n_hh; ++l) {
      so.w[l] = q->woff[l + 1];
      a.off_bh[l] = q->boff[l + 1];
    }
    square_weights_kernel<<<grid1((int64_t)q->cfg.n_members * n_hh * mlptc::H * mlptc::H), 256, 0, s>>>(
        q->params, q->P, q->cfg.n_members, n_hh, so, q->whh);
    SDE_CUDA_TRY(cudaGetLastError());
    a.X = X;
    a.params = q->params;
    a.P = q->P;
    a.B = B;
    a.n_in = q->cfg.n_in;
    a.n_hh = n_hh;
    a.off_w0 = q->woff[0];
    a.off_b0 = q->boff[0];
    a.off_wo = q->woff[q->L - 1];
    a.off_bo = q->boff[q->L - 1];
    a.out = q->out;
    a.out_stride = q->cfg.max_batch;
    a.err = q->err;
    const dim3 grid((unsigned)((B + mlptc::BM - 1) / mlptc::BM), (unsigned)q->cfg.n_members);
    mlptc::mlp_fwd_tc_kernel<<<grid, mlptc::THREADS, mlptc::SMEM_BYTES, s>>>(q->map_whh, a);
    SDE_CUDA_TRY(cudaGetLastError());
  } else {
    for (int mm = 0; mm < q->cfg.n_members; ++mm) {
      sde_status st = mlp_forward_member(q, mm, X, B, q->out + (int64_t)mm * q->cfg.max_batch, s);
      if (st != SDE_OK) return st;
    }
  }
  ensemble_stats_kernel<<<grid1(B), 256, 0, s>>>(q->out, q->cfg.n_members, q->cfg.max_batch, B, mean, spread);
  SDE_CUDA_TRY(cudaGetLastError());
  return SDE_OK;
}

sde_status sde_mlp_grad(sde_mlp *q, int32_t member, const float *X, const float *y, int64_t B, float *grad,
                        float *loss, void *stream) {
  clear_error();
  SDE_CHECK_ARG(q != nullptr, "mlp is NULL");
  SDE_CHECK_ARG(member >= 0 && member < q->cfg.n_members, "member out of range");
  SDE_CHECK_ARG(B >= 1 && B <= q->cfg.max_batch, "batch must be in [1, max_batch]");
  SDE_CHECK_ARG(X && y && grad, "X, y and grad must be non-NULL");
  return mlp_grad_member(q, member, X, y, B, grad, loss, (cudaStream_t)stream);
}

sde_status sde_mlp_use_tensor_cores(sde_mlp *q, int32_t enable) {
  clear_error();
  SDE_CHECK_ARG(q != nullptr, "mlp is NULL");
  if (enable && !q->tc) {
    set_error("the tensor-core forward needs hidden == 256, 2..8 hidden layers and n_in <= 8");
    return SDE_ERR_UNSUPPORTED;
  }
  q->use_tc = enable != 0;
  return SDE_OK;
}

sde_status sde_mlp_check(sde_mlp *q) {
  clear_error();
  SDE_CHECK_ARG(q != nullptr, "mlp is NULL");
  SDE_CUDA_TRY(cudaDeviceSynchronize());
  uint32_t err = 0;
  SDE_CUDA_TRY(cudaMemcpy(&err, q->err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (err) SDE_CUDA_TRY(cudaMemset(q->err, 0, sizeof(uint32_t)));
  if (err & kErrTimeout) {
    set_error("a bounded device wait of the tensor-core forward expired");
    return SDE_ERR_TIMEOUT;
  }
  return SDE_OK;
}

sde_status sde_mlp_set_lr(sde_mlp *q, float lr) {
  clear_error();
  SDE_CHECK_ARG(q != nullptr && lr > 0.0f, "mlp must be non-NULL and lr > 0");
  q->cfg.lr = lr;
  return SDE_OK;
}

static sde_status mlp_train(sde_mlp *q, const float *X, const float *y, int64_t B, float *loss, void *stream,
                            bool per_member) {
  clear_error();
  SDE_CHECK_ARG(q != nullptr, "mlp is NULL");
  SDE_CHECK_ARG(B >= 1 && B <= q->cfg.max_batch, "batch must be in [1, max_batch]");
  SDE_CHECK_ARG(X && y, "X and y must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  for (int mm = 0; mm < q->cfg.n_members; ++mm) {
    const int64_t xo = per_member ? (int64_t)mm * B * q->cfg.n_in : 0;
    const int64_t yo = per_member ? (int64_t)mm * B : 0;
    sde_status st = mlp_grad_member(q, mm, X + xo, y + yo, B, q->grad + (int64_t)mm * q->P,
                                    loss ? loss + mm : nullptr, s);
    if (st != SDE_OK) return st;
  }
  q->step += 1;
  const double b1 = q->cfg.beta1, b2 = q->cfg.beta2;
  const double c1 = 1.0 - pow(b1, (double)q->step), c2 = 1.0 - pow(b2, (double)q->step);
  // Adam with the bias corrections folded into the step size and epsilon:
  // p -= lr * (m / c1) / (sqrt(v / c2) + eps) = (lr sqrt(c2) / c1) m / (sqrt(v) + eps sqrt(c2))
  const float lr_t = (float)(q->cfg.lr * sqrt(c2) / c1);
  const float eps_t = (float)(q->cfg.eps * sqrt(c2));
  const int64_t n = q->P * q->cfg.n_members;
  adam_kernel<<<grid1(n), 256, 0, s>>>(q->params, q->grad, q->m, q->v, n, lr_t, (float)b1, (float)b2, eps_t);
  SDE_CUDA_TRY(cudaGetLastError());
  return SDE_OK;
}

sde_status sde_mlp_train_step(sde_mlp *q, const float *X, const float *y, int64_t B, float *loss, void *stream) {
  return mlp_train(q, X, y, B, loss, stream, false);
}

sde_status sde_mlp_train_step_members(sde_mlp *q, const float *X, const float *y, int64_t B, float *loss,
                                      void *stream) {
  return mlp_train(q, X, y, B, loss, stream, true);
}

}  // extern "C"
