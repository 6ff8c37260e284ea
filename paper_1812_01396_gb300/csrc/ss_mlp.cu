// Warm-start network: a 3-layer MLP (E, k) -> surface Green's function of a
// lead, trained and run by the library's own kernels.
//
// Layers 19 -> W -> W -> n_out with SiLU between them, mean-squared loss,
// Adam.  FP32 master weights; every GEMM reads BF16 copies of the weights and
// of the activations and accumulates in FP32 (the "BF16 weights" of the
// warm-start workload).  The GEMMs are small (about 34 MFLOP per sample), so
// they run as tiled SIMT kernels.
//
// Layout: every matrix row-major; W1 (W x n_in), W2 (W x W), W3 (n_out x W);
// activations (B x features).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "splitsolve.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int T = 64, TK = 16, NT = 256;

// C (M x N, fp32, ldc) = op(A) op(B) [+ bias (N)] [+ beta C]; A and B bf16.
// ta: op(A) = A^T with A stored (K x M); tb: op(B) = B^T with B stored (N x K).
__global__ void __launch_bounds__(NT) mlp_gemm_kernel(int M, int N, int K, const bf16* __restrict__ A, int lda,
                                                      int ta, const bf16* __restrict__ B, int ldb, int tb,
                                                      float* __restrict__ C, int ldc, const float* __restrict__ bias,
                                                      float beta) {
  __shared__ float As[TK][T + 1];
  __shared__ float Bs[TK][T + 1];
  const int row0 = blockIdx.y * T, col0 = blockIdx.x * T;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = tid; e < T * TK; e += NT) {
      int r, kk;
      if (ta) { kk = e / T; r = e % T; } else { r = e / TK; kk = e % TK; }
      const int gi = row0 + r, gk = k0 + kk;
      float v = 0.f;
      if (gi < M && gk < K) v = __bfloat162float(ta ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk]);
      As[kk][r] = v;
    }
    for (int e = tid; e < T * TK; e += NT) {
      int c, kk;
      if (tb) { c = e / TK; kk = e % TK; } else { kk = e / T; c = e % T; }
      const int gj = col0 + c, gk = k0 + kk;
      float v = 0.f;
      if (gj < N && gk < K) v = __bfloat162float(tb ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj]);
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c >= N) continue;
      float v = acc[i][j];
      if (bias) v += bias[c];
      if (beta != 0.f) v += beta * C[(size_t)r * ldc + c];
      C[(size_t)r * ldc + c] = v;
    }
  }
}

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + __expf(-x)); }

// a = silu(h) (fp32 and bf16 copies)
__global__ void silu_fwd_kernel(const float* h, float* a, bf16* ab, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = h[i] * sigm(h[i]);
  a[i] = v;
  ab[i] = __float2bfloat16(v);
}

// dh = da * silu'(h), stored fp32 and bf16
__global__ void silu_bwd_kernel(const float* da, const float* h, float* dh, bf16* dhb, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float s = sigm(h[i]);
  const float v = da[i] * s * (1.f + h[i] * (1.f - s));
  dh[i] = v;
  dhb[i] = __float2bfloat16(v);
}

// dy = 2 (y - t) / (B n_out) in bf16; per-block partial sums of (y - t)^2
__global__ void mse_kernel(const float* y, const float* t, bf16* dyb, float* dyf, double* partial, int n, float inv) {
  __shared__ double red[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < n) {
    const float d = y[i] - t[i];
    s = (double)d * d;
    const float g = 2.f * d * inv;
    dyb[i] = __float2bfloat16(g);
    dyf[i] = g;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// db[j] = sum_b d[b][j]
__global__ void colsum_kernel(const float* d, float* db, int B, int N) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += d[(size_t)b * N + j];
  db[j] = s;
}

__global__ void to_bf16_kernel(const float* x, bf16* y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16(x[i]);
}

// Adam with bias correction on the FP32 master weights, refreshing the BF16 copy
__global__ void adam_kernel(float* w, bf16* wb, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] -= upd;
  if (wb) wb[i] = __float2bfloat16(w[i]);
}

int blocks(long long n) { return (int)((n + 255) / 256); }

}  // namespace

struct ss_mlp {
  int n_in, width, n_out, max_batch;
  // params: W1 b1 W2 b2 W3 b3 (fp32 master), bf16 copies of W1 W2 W3
  float* p[6] = {nullptr};
  float* g[6] = {nullptr};
  float* m[6] = {nullptr};
  float* v[6] = {nullptr};
  bf16* wb[3] = {nullptr};
  size_t count[6];
  // activations
  bf16* xb = nullptr;
  float *h1, *a1, *h2, *a2, *y, *dy, *da2, *dh2, *da1, *dh1;
  bf16 *a1b, *a2b, *dyb, *dh2b, *dh1b;
  double* partial = nullptr;
  int step = 0;
  cudaStream_t st = nullptr;
  std::string err;
};

namespace {

void gemm(ss_mlp* n, int M, int N, int K, const bf16* A, int lda, int ta, const bf16* B, int ldb, int tb, float* C,
          int ldc, const float* bias, float beta) {
  dim3 grid((N + T - 1) / T, (M + T - 1) / T);
  mlp_gemm_kernel<<<grid, NT, 0, n->st>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, bias, beta);
}

// forward for a batch already in n->xb (bf16, B x n_in); output n->y
void forward(ss_mlp* n, int B) {
  const int W = n->width;
  gemm(n, B, W, n->n_in, n->xb, n->n_in, 0, n->wb[0], n->n_in, 1, n->h1, W, n->p[1], 0.f);
  silu_fwd_kernel<<<blocks((long long)B * W), 256, 0, n->st>>>(n->h1, n->a1, n->a1b, B * W);
  gemm(n, B, W, W, n->a1b, W, 0, n->wb[1], W, 1, n->h2, W, n->p[3], 0.f);
  silu_fwd_kernel<<<blocks((long long)B * W), 256, 0, n->st>>>(n->h2, n->a2, n->a2b, B * W);
  gemm(n, B, n->n_out, W, n->a2b, W, 0, n->wb[2], W, 1, n->y, n->n_out, n->p[5], 0.f);
}

// backward from n->dyb / n->dy (B x n_out) into n->g[*]
void backward(ss_mlp* n, int B) {
  const int W = n->width, O = n->n_out;
  // dW3 = dy^T a2 ; db3 = colsum(dy) ; da2 = dy W3
  gemm(n, O, W, B, n->dyb, O, 1, n->a2b, W, 0, n->g[4], W, nullptr, 0.f);
  colsum_kernel<<<blocks(O), 256, 0, n->st>>>(n->dy, n->g[5], B, O);
  gemm(n, B, W, O, n->dyb, O, 0, n->wb[2], W, 0, n->da2, W, nullptr, 0.f);
  silu_bwd_kernel<<<blocks((long long)B * W), 256, 0, n->st>>>(n->da2, n->h2, n->dh2, n->dh2b, B * W);
  gemm(n, W, W, B, n->dh2b, W, 1, n->a1b, W, 0, n->g[2], W, nullptr, 0.f);
  colsum_kernel<<<blocks(W), 256, 0, n->st>>>(n->dh2, n->g[3], B, W);
  gemm(n, B, W, W, n->dh2b, W, 0, n->wb[1], W, 0, n->da1, W, nullptr, 0.f);
  silu_bwd_kernel<<<blocks((long long)B * W), 256, 0, n->st>>>(n->da1, n->h1, n->dh1, n->dh1b, B * W);
  gemm(n, W, n->n_in, B, n->dh1b, W, 1, n->xb, n->n_in, 0, n->g[0], n->n_in, nullptr, 0.f);
  colsum_kernel<<<blocks(W), 256, 0, n->st>>>(n->dh1, n->g[1], B, W);
}

int mlp_fail(ss_mlp* n, int code, const std::string& msg) {
  if (n) n->err = msg;
  return code;
}

}  // namespace

extern "C" {

int ss_mlp_create(ss_mlp** out, int n_in, int width, int n_out, int max_batch, unsigned long long seed, void* stream) {
  if (!out || n_in < 1 || width < 1 || n_out < 1 || max_batch < 1) return SS_ERR_ARG;
  *out = nullptr;
  ss_mlp* n = new ss_mlp();
  n->n_in = n_in; n->width = width; n->n_out = n_out; n->max_batch = max_batch;
  n->st = (cudaStream_t)stream;
  const size_t cnt[6] = {(size_t)width * n_in, (size_t)width, (size_t)width * width, (size_t)width,
                         (size_t)n_out * width, (size_t)n_out};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) {
    n->count[i] = cnt[i];
    e = cudaMalloc(&n->p[i], cnt[i] * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->g[i], cnt[i] * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->m[i], cnt[i] * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->v[i], cnt[i] * 4);
    if (e == cudaSuccess) e = cudaMemset(n->m[i], 0, cnt[i] * 4);
    if (e == cudaSuccess) e = cudaMemset(n->v[i], 0, cnt[i] * 4);
  }
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc(&n->wb[i], cnt[2 * i] * 2);
  const size_t BW = (size_t)max_batch * width, BO = (size_t)max_batch * n_out;
  float** f32[] = {&n->h1, &n->a1, &n->h2, &n->a2, &n->da2, &n->dh2, &n->da1, &n->dh1};
  for (float** q : f32) if (e == cudaSuccess) e = cudaMalloc(q, BW * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->y, BO * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->dy, BO * 4);
  bf16** b16[] = {&n->a1b, &n->a2b, &n->dh2b, &n->dh1b};
  for (bf16** q : b16) if (e == cudaSuccess) e = cudaMalloc(q, BW * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->dyb, BO * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->xb, (size_t)max_batch * n_in * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->partial, (size_t)blocks((long long)BO) * sizeof(double));
  if (e != cudaSuccess) { cudaGetLastError(); ss_mlp_destroy(n); return SS_ERR_OOM; }
  // deterministic init on the host: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a 64-bit LCG, zero biases
  unsigned long long st = seed * 6364136223846793005ull + 1442695040888963407ull;
  const int fan[3] = {n_in, width, width};
  for (int l = 0; l < 3; ++l) {
    std::vector<float> w(cnt[2 * l]), b(cnt[2 * l + 1], 0.f);
    const float lim = 1.f / std::sqrt((float)fan[l]);
    for (auto& x : w) {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      x = lim * (2.f * (float)((st >> 40) & 0xFFFFFF) / 16777216.f - 1.f);
    }
    if (e == cudaSuccess) e = cudaMemcpy(n->p[2 * l], w.data(), w.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(n->p[2 * l + 1], b.data(), b.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      to_bf16_kernel<<<blocks((long long)w.size()), 256, 0, n->st>>>(n->p[2 * l], n->wb[l], (int)w.size());
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->st);
  if (e != cudaSuccess) { ss_mlp_destroy(n); return SS_ERR_CUDA; }
  *out = n;
  return SS_OK;
}

int ss_mlp_destroy(ss_mlp* n) {
  if (!n) return SS_OK;
  for (int i = 0; i < 6; ++i) { cudaFree(n->p[i]); cudaFree(n->g[i]); cudaFree(n->m[i]); cudaFree(n->v[i]); }
  for (int i = 0; i < 3; ++i) cudaFree(n->wb[i]);
  float* f32[] = {n->h1, n->a1, n->h2, n->a2, n->da2, n->dh2, n->da1, n->dh1, n->y, n->dy};
  for (float* q : f32) cudaFree(q);
  bf16* b16[] = {n->a1b, n->a2b, n->dh2b, n->dh1b, n->dyb, n->xb};
  for (bf16* q : b16) cudaFree(q);
  cudaFree(n->partial);
  delete n;
  return SS_OK;
}

// params: host or device arrays W1 b1 W2 b2 W3 b3 (fp32) in the order above
int ss_mlp_set_params(ss_mlp* n, const float* const* params, int device_ptrs) {
  if (!n || !params) return SS_ERR_ARG;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 6 && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(n->p[i], params[i], n->count[i] * 4, device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        n->st);
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    to_bf16_kernel<<<blocks((long long)n->count[2 * l]), 256, 0, n->st>>>(n->p[2 * l], n->wb[l], (int)n->count[2 * l]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->st);
  return e == cudaSuccess ? SS_OK : mlp_fail(n, SS_ERR_CUDA, cudaGetErrorString(e));
}

// copy the FP32 master params (or, which = 1, the last gradients) to host arrays
int ss_mlp_get(ss_mlp* n, int which, float* const* out) {
  if (!n || !out) return SS_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(n->st);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i)
    e = cudaMemcpy(out[i], which ? n->g[i] : n->p[i], n->count[i] * 4, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SS_OK : mlp_fail(n, SS_ERR_CUDA, cudaGetErrorString(e));
}

// y (B x n_out, device fp32) = MLP(x), x (B x n_in, device fp32)
int ss_mlp_forward(ss_mlp* n, int B, const float* x, float* y) {
  if (!n || B < 1 || B > n->max_batch || !x) return SS_ERR_ARG;
  to_bf16_kernel<<<blocks((long long)B * n->n_in), 256, 0, n->st>>>(x, n->xb, B * n->n_in);
  forward(n, B);
  cudaError_t e = cudaSuccess;
  if (y) e = cudaMemcpyAsync(y, n->y, (size_t)B * n->n_out * 4, cudaMemcpyDeviceToDevice, n->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? SS_OK : mlp_fail(n, SS_ERR_CUDA, cudaGetErrorString(e));
}

// One step: forward, mean-squared loss against t, backward; with lr > 0 also
// an Adam update (beta1 0.9, beta2 0.999, eps 1e-8).  Device x, t; *loss on host.
int ss_mlp_train_step(ss_mlp* n, int B, const float* x, const float* t, float lr, double* loss) {
  if (!n || B < 1 || B > n->max_batch || !x || !t) return SS_ERR_ARG;
  to_bf16_kernel<<<blocks((long long)B * n->n_in), 256, 0, n->st>>>(x, n->xb, B * n->n_in);
  forward(n, B);
  const int BO = B * n->n_out;
  const int nb = blocks(BO);
  mse_kernel<<<nb, 256, 0, n->st>>>(n->y, t, n->dyb, n->dy, n->partial, BO, 1.f / (float)BO);
  backward(n, B);
  if (lr > 0.f) {
    ++n->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
    for (int i = 0; i < 6; ++i)
      adam_kernel<<<blocks((long long)n->count[i]), 256, 0, n->st>>>(n->p[i], (i % 2 == 0) ? n->wb[i / 2] : nullptr, n->g[i],
                                                                   n->m[i], n->v[i], (int)n->count[i], lr, b1, b2, c1, c2,
                                                                   1e-8f);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && loss) {
    std::vector<double> part(nb);
    e = cudaMemcpyAsync(part.data(), n->partial, nb * sizeof(double), cudaMemcpyDeviceToHost, n->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->st);
    double s = 0.0;
    for (double q : part) s += q;
    *loss = s / (double)BO;
  }
  return e == cudaSuccess ? SS_OK : mlp_fail(n, SS_ERR_CUDA, cudaGetErrorString(e));
}

const char* ss_mlp_last_error(const ss_mlp* n) { return n ? n->err.c_str() : ""; }

}  // extern "C"

namespace ss {
cudaStream_t mlp_stream(const ss_mlp* n) { return n->st; }
void mlp_dims(const ss_mlp* n, int* n_in, int* n_out, int* max_batch) {
  *n_in = n->n_in;
  *n_out = n->n_out;
  *max_batch = n->max_batch;
}
}  // namespace ss
