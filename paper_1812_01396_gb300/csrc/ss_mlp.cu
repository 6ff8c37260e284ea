// Warm-start network: a 3-layer MLP (E, k) -> surface Green's function of a
// lead, trained and run by the library's own kernels.
//
// Layers 19 -> W -> W -> n_out with SiLU between them, mean-squared loss,
// Adam.  FP32 master weights; every GEMM reads BF16 copies of the weights and
// of the activations and accumulates in FP32 (the "BF16 weights" of the
// warm-start workload).
//
// The GEMMs run on the tcgen05 tensor cores (kind::f16, BF16 x BF16 -> FP32 in
// TMEM) when the width and n_out are multiples of 8: one CTA per 128 x 128
// output tile, TMA loads of 64-wide K slices into a 4-stage ring, one thread
// issuing the MMAs, four epilogue warps adding the bias (and beta C).  Both
// operands are K-major; the backward products, whose contraction runs along
// the batch or along the output features, read transposed BF16 copies made by
// a tiled transpose kernel (the weights' copies are refreshed after each Adam
// step).  Other widths use a tiled SIMT kernel with the same rounding points.
//
// Layout: every matrix row-major; W1 (W x n_in), W2 (W x W), W3 (n_out x W);
// activations (B x features).  The BF16 copies of x and W1 have a row stride of
// n_in rounded up to 8 (16-byte rows for the tensor maps).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "splitsolve.h"
#include "ss_tc.h"
#include "ss_tcutil.cuh"

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

// ---- tensor-core GEMM: C (M x N, fp32, ldc) = A B^T [+ bias (N)] [+ beta C],
// A (M x K) and B (N x K) BF16, K-major, read through the tensor maps ma / mb
// (zero fill past M, N and K).
constexpr int TBM = 128, TBN = 128, TBK = 64, TSTAGES = 4;
constexpr int TTHREADS = 192;  // warp 0: TMA, warp 1: MMA + TMEM, warps 2-5: epilogue
constexpr uint32_t TA_BYTES = TBM * TBK * 2, TB_BYTES = TBN * TBK * 2, TSTAGE_BYTES = TA_BYTES + TB_BYTES;
constexpr uint32_t TTMEM_COLS = TBN;
// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = 128.
constexpr uint32_t TIDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                            ((uint32_t)(TBM >> 4) << 24);
constexpr size_t TSMEM = (size_t)TSTAGES * TSTAGE_BYTES + 1024;

__global__ void __launch_bounds__(TTHREADS, 1) mlp_tc_kernel(const __grid_constant__ CUtensorMap ma,
                                                             const __grid_constant__ CUtensorMap mb, int M, int N,
                                                             int K, float* __restrict__ C, int ldc,
                                                             const float* __restrict__ bias, float beta, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[TSTAGES];
  __shared__ __align__(8) uint64_t empty_bar[TSTAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const int ktiles = (K + TBK - 1) / TBK;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < TSTAGES; ++i) { ss::mbar_init(&full_bar[i], 1); ss::mbar_init(&empty_bar[i], 1); }
    ss::mbar_init(&acc_bar, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ss::smem_u32(&tmem_base)),
                 "r"(TTMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (warp == 0 && lane == 0) {
    for (int kt = 0; kt < ktiles; ++kt) {
      const int st = kt % TSTAGES;
      const uint32_t ph = (kt / TSTAGES) & 1;
      if (!ss::mbar_wait(&empty_bar[st], ph ^ 1)) { s_fail = 1; break; }
      unsigned char* sa = smem + st * TSTAGE_BYTES;
      ss::mbar_expect_tx(&full_bar[st], TSTAGE_BYTES);
      ss::tma_load_2d(sa, &ma, &full_bar[st], kt * TBK, m0);
      ss::tma_load_2d(sa + TA_BYTES, &mb, &full_bar[st], kt * TBK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    bool ok = true;
    for (int kt = 0; kt < ktiles; ++kt) {
      const int st = kt % TSTAGES;
      const uint32_t ph = (kt / TSTAGES) & 1;
      if (!ss::mbar_wait(&full_bar[st], ph)) { ok = false; s_fail = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* sa = smem + st * TSTAGE_BYTES;
      const uint64_t da = ss::smem_desc(sa), db = ss::smem_desc(sa + TA_BYTES);
#pragma unroll
      for (int k = 0; k < TBK / 16; ++k)
        ss::mma_bf16(tmem, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), TIDESC, (kt | k) != 0);
      ss::mma_commit(&empty_bar[st]);
    }
    if (ok) ss::mma_commit(&acc_bar);
    else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ss::smem_u32(&acc_bar)) : "memory");
  } else if (warp >= 2) {
    const bool ok = ss::mbar_wait(&acc_bar, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int q = warp & 3;  // TMEM lane quarter this warp may read
    const int row = m0 + q * 32 + lane;
    if (ok && !s_fail) {
#pragma unroll 1
      for (int c = 0; c < TBN / 32; ++c) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < M) {
          float* crow = C + (size_t)row * ldc;
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int col = n0 + c * 32 + e;
            if (col < N) {
              float x = __uint_as_float(v[e]);
              if (bias) x += bias[col];
              if (beta != 0.f) x += beta * crow[col];
              crow[col] = x;
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (s_fail && threadIdx.x == 0 && err) atomicExch(err, 1);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TTMEM_COLS) : "memory");
  }
}

// out (Cc x R, row stride ldo) = in^T, in (R x Cc, row stride ldi); 32 x 32 tiles through shared memory
__global__ void transpose_bf16_kernel(const bf16* __restrict__ in, int ldi, int R, int Cc, bf16* __restrict__ out,
                                      int ldo) {
  __shared__ bf16 tile[32][34];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < Cc) tile[i][threadIdx.x] = in[(size_t)r * ldi + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < Cc && r < R) out[(size_t)c * ldo + r] = tile[threadIdx.x][i];
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

// y (row stride ldy) = bf16(x), x dense with `cols` columns
__global__ void to_bf16_kernel(const float* x, bf16* y, int n, int cols, int ldy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[(size_t)(i / cols) * ldy + i % cols] = __float2bfloat16(x[i]);
}

// Adam with bias correction on the FP32 master weights, refreshing the BF16 copy
__global__ void adam_kernel(float* w, bf16* wb, int cols, int ldw, const float* g, float* m, float* v, int n, float lr,
                            float b1, float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] -= upd;
  if (wb) wb[(size_t)(i / cols) * ldw + i % cols] = __float2bfloat16(w[i]);
}

int blocks(long long n) { return (int)((n + 255) / 256); }

}  // namespace

struct ss_mlp {
  int n_in, width, n_out, max_batch;
  int ldx;   // row stride of the BF16 copies of x and W1: n_in rounded up to 8
  int bp;    // row stride of the transposed activations: max_batch rounded up to 8
  int tc = 0;  // GEMMs on the tensor cores
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
  // transposed BF16 copies for the tensor-core backward: x^T, a1^T, a2^T, dh2^T, dh1^T,
  // dy^T (features x bp) and W2^T (W x W), W3^T (W x n_out)
  bf16 *xT = nullptr, *a1T = nullptr, *a2T = nullptr, *dh2T = nullptr, *dh1T = nullptr, *dyT = nullptr;
  bf16 *w2T = nullptr, *w3T = nullptr;
  int* derr = nullptr;  // set by a tensor-core GEMM whose pipeline wait timed out
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

// C = A B^T (+ bias), A (M x K, lda) and B (N x K, ldb) K-major, on the tensor cores
cudaError_t gemm_tc(ss_mlp* n, int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc,
                    const float* bias) {
  CUtensorMap ma, mb;
  cudaError_t e = ss::encode_kmajor_map(&ma, A, M, K, TBM, lda);
  if (e == cudaSuccess) e = ss::encode_kmajor_map(&mb, B, N, K, TBN, ldb);
  if (e != cudaSuccess) return e;
  dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM);
  mlp_tc_kernel<<<grid, TTHREADS, TSMEM, n->st>>>(ma, mb, M, N, K, C, ldc, bias, 0.f, n->derr);
  return cudaGetLastError();
}

void transpose(ss_mlp* n, const bf16* in, int ldi, int R, int Cc, bf16* out, int ldo) {
  dim3 grid((Cc + 31) / 32, (R + 31) / 32);
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, n->st>>>(in, ldi, R, Cc, out, ldo);
}

// transposed BF16 copies of W2 and W3 for the tensor-core backward
void refresh_wT(ss_mlp* n) {
  if (!n->tc) return;
  const int W = n->width, O = n->n_out;
  transpose(n, n->wb[1], W, W, W, n->w2T, W);
  transpose(n, n->wb[2], W, O, W, n->w3T, O);
}

// forward for a batch already in n->xb (bf16, B x n_in, row stride ldx); output n->y
cudaError_t forward(ss_mlp* n, int B) {
  const int W = n->width, O = n->n_out;
  cudaError_t e = cudaSuccess;
  if (n->tc) e = gemm_tc(n, B, W, n->n_in, n->xb, n->ldx, n->wb[0], n->ldx, n->h1, W, n->p[1]);
  else gemm(n, B, W, n->n_in, n->xb, n->ldx, 0, n->wb[0], n->ldx, 1, n->h1, W, n->p[1], 0.f);
  silu_fwd_kernel<<<blocks((long long)B * W), 256, 0, n->st>>>(n->h1, n->a1, n->a1b, B * W);
  if (n->tc) { if (e == cudaSuccess) e = gemm_tc(n, B, W, W, n->a1b, W, n->wb[1], W, n->h2, W, n->p[3]); }
  else gemm(n, B, W, W, n->a1b, W, 0, n->wb[1], W, 1, n->h2, W, n->p[3], 0.f);
  silu_fwd_kernel<<<blocks((long long)B * W), 256, 0, n->st>>>(n->h2, n->a2, n->a2b, B * W);
  if (n->tc) { if (e == cudaSuccess) e = gemm_tc(n, B, O, W, n->a2b, W, n->wb[2], W, n->y, O, n->p[5]); }
  else gemm(n, B, O, W, n->a2b, W, 0, n->wb[2], W, 1, n->y, O, n->p[5], 0.f);
  return e;
}

// backward from n->dyb / n->dy (B x n_out) into n->g[*]
cudaError_t backward(ss_mlp* n, int B) {
  const int W = n->width, O = n->n_out, bp = n->bp;
  cudaError_t e = cudaSuccess;
  // dW3 = dy^T a2 ; db3 = colsum(dy) ; da2 = dy W3
  if (n->tc) {
    transpose(n, n->dyb, O, B, O, n->dyT, bp);
    transpose(n, n->a2b, W, B, W, n->a2T, bp);
    e = gemm_tc(n, O, W, B, n->dyT, bp, n->a2T, bp, n->g[4], W, nullptr);
  } else {
    gemm(n, O, W, B, n->dyb, O, 1, n->a2b, W, 0, n->g[4], W, nullptr, 0.f);
  }
  colsum_kernel<<<blocks(O), 256, 0, n->st>>>(n->dy, n->g[5], B, O);
  if (n->tc) { if (e == cudaSuccess) e = gemm_tc(n, B, W, O, n->dyb, O, n->w3T, O, n->da2, W, nullptr); }
  else gemm(n, B, W, O, n->dyb, O, 0, n->wb[2], W, 0, n->da2, W, nullptr, 0.f);
  silu_bwd_kernel<<<blocks((long long)B * W), 256, 0, n->st>>>(n->da2, n->h2, n->dh2, n->dh2b, B * W);
  // dW2 = dh2^T a1 ; db2 ; da1 = dh2 W2
  if (n->tc) {
    transpose(n, n->dh2b, W, B, W, n->dh2T, bp);
    transpose(n, n->a1b, W, B, W, n->a1T, bp);
    if (e == cudaSuccess) e = gemm_tc(n, W, W, B, n->dh2T, bp, n->a1T, bp, n->g[2], W, nullptr);
  } else {
    gemm(n, W, W, B, n->dh2b, W, 1, n->a1b, W, 0, n->g[2], W, nullptr, 0.f);
  }
  colsum_kernel<<<blocks(W), 256, 0, n->st>>>(n->dh2, n->g[3], B, W);
  if (n->tc) { if (e == cudaSuccess) e = gemm_tc(n, B, W, W, n->dh2b, W, n->w2T, W, n->da1, W, nullptr); }
  else gemm(n, B, W, W, n->dh2b, W, 0, n->wb[1], W, 0, n->da1, W, nullptr, 0.f);
  silu_bwd_kernel<<<blocks((long long)B * W), 256, 0, n->st>>>(n->da1, n->h1, n->dh1, n->dh1b, B * W);
  // dW1 = dh1^T x ; db1
  if (n->tc) {
    transpose(n, n->dh1b, W, B, W, n->dh1T, bp);
    transpose(n, n->xb, n->ldx, B, n->n_in, n->xT, bp);
    if (e == cudaSuccess) e = gemm_tc(n, W, n->n_in, B, n->dh1T, bp, n->xT, bp, n->g[0], n->n_in, nullptr);
  } else {
    gemm(n, W, n->n_in, B, n->dh1b, W, 1, n->xb, n->ldx, 0, n->g[0], n->n_in, nullptr, 0.f);
  }
  colsum_kernel<<<blocks(W), 256, 0, n->st>>>(n->dh1, n->g[1], B, W);
  return e;
}

// BF16 copy of master parameter i (W1, W2 or W3) with its row stride
void refresh_wb(ss_mlp* n, int l) {
  const int cols = l == 0 ? n->n_in : n->width;
  const int ld = l == 0 ? n->ldx : cols;
  to_bf16_kernel<<<blocks((long long)n->count[2 * l]), 256, 0, n->st>>>(n->p[2 * l], n->wb[l], (int)n->count[2 * l],
                                                                       cols, ld);
}

// reports (and clears) a timed-out tensor-core pipeline wait; the stream is synchronised
cudaError_t check_derr(ss_mlp* n) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, n->derr, sizeof(int), cudaMemcpyDeviceToHost, n->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->st);
  if (e == cudaSuccess && h) {
    cudaMemsetAsync(n->derr, 0, sizeof(int), n->st);
    n->err = "tensor-core GEMM: a pipeline wait timed out";
    return cudaErrorLaunchTimeout;
  }
  return e;
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
  n->ldx = (n_in + 7) / 8 * 8;
  n->bp = (max_batch + 7) / 8 * 8;
  n->tc = (width % 8 == 0 && n_out % 8 == 0) ? 1 : 0;
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
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    const size_t c = i == 0 ? (size_t)width * n->ldx : cnt[2 * i];
    e = cudaMalloc(&n->wb[i], c * 2);
    if (e == cudaSuccess) e = cudaMemset(n->wb[i], 0, c * 2);
  }
  const size_t BW = (size_t)max_batch * width, BO = (size_t)max_batch * n_out;
  float** f32[] = {&n->h1, &n->a1, &n->h2, &n->a2, &n->da2, &n->dh2, &n->da1, &n->dh1};
  for (float** q : f32) if (e == cudaSuccess) e = cudaMalloc(q, BW * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->y, BO * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->dy, BO * 4);
  bf16** b16[] = {&n->a1b, &n->a2b, &n->dh2b, &n->dh1b};
  for (bf16** q : b16) if (e == cudaSuccess) e = cudaMalloc(q, BW * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->dyb, BO * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->xb, (size_t)max_batch * n->ldx * 2);
  if (e == cudaSuccess) e = cudaMemset(n->xb, 0, (size_t)max_batch * n->ldx * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->partial, (size_t)blocks((long long)BO) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&n->derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->derr, 0, sizeof(int));
  if (n->tc) {
    const size_t bp = n->bp;
    bf16** t16[] = {&n->a1T, &n->a2T, &n->dh2T, &n->dh1T};
    for (bf16** q : t16) if (e == cudaSuccess) e = cudaMalloc(q, (size_t)width * bp * 2);
    if (e == cudaSuccess) e = cudaMalloc(&n->xT, (size_t)n_in * bp * 2);
    if (e == cudaSuccess) e = cudaMalloc(&n->dyT, (size_t)n_out * bp * 2);
    if (e == cudaSuccess) e = cudaMalloc(&n->w2T, (size_t)width * width * 2);
    if (e == cudaSuccess) e = cudaMalloc(&n->w3T, (size_t)width * n_out * 2);
    if (e == cudaSuccess) {
      e = cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TSMEM);
      if (e != cudaSuccess) { cudaGetLastError(); ss_mlp_destroy(n); return SS_ERR_CUDA; }
    }
  }
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
      refresh_wb(n, l);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    refresh_wT(n);
    e = cudaGetLastError();
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
  bf16* b16[] = {n->a1b, n->a2b, n->dh2b, n->dh1b, n->dyb, n->xb, n->xT, n->a1T, n->a2T, n->dh2T, n->dh1T, n->dyT,
                 n->w2T, n->w3T};
  for (bf16* q : b16) cudaFree(q);
  cudaFree(n->partial);
  cudaFree(n->derr);
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
    refresh_wb(n, l);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    refresh_wT(n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->st);
  return e == cudaSuccess ? SS_OK : mlp_fail(n, SS_ERR_CUDA, cudaGetErrorString(e));
}

// copy the FP32 master params (or, which = 1, the last gradients) to host arrays
int ss_mlp_get(ss_mlp* n, int which, float* const* out) {
  if (!n || !out) return SS_ERR_ARG;
  cudaError_t e = check_derr(n);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i)
    e = cudaMemcpy(out[i], which ? n->g[i] : n->p[i], n->count[i] * 4, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SS_OK : mlp_fail(n, SS_ERR_CUDA, cudaGetErrorString(e));
}

// y (B x n_out, device fp32) = MLP(x), x (B x n_in, device fp32)
int ss_mlp_forward(ss_mlp* n, int B, const float* x, float* y) {
  if (!n || B < 1 || B > n->max_batch || !x) return SS_ERR_ARG;
  to_bf16_kernel<<<blocks((long long)B * n->n_in), 256, 0, n->st>>>(x, n->xb, B * n->n_in, n->n_in, n->ldx);
  cudaError_t e = forward(n, B);
  if (e == cudaSuccess && y) e = cudaMemcpyAsync(y, n->y, (size_t)B * n->n_out * 4, cudaMemcpyDeviceToDevice, n->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? SS_OK : mlp_fail(n, SS_ERR_CUDA, cudaGetErrorString(e));
}

// One step: forward, mean-squared loss against t, backward; with lr > 0 also
// an Adam update (beta1 0.9, beta2 0.999, eps 1e-8).  Device x, t; *loss on host.
int ss_mlp_train_step(ss_mlp* n, int B, const float* x, const float* t, float lr, double* loss) {
  if (!n || B < 1 || B > n->max_batch || !x || !t) return SS_ERR_ARG;
  to_bf16_kernel<<<blocks((long long)B * n->n_in), 256, 0, n->st>>>(x, n->xb, B * n->n_in, n->n_in, n->ldx);
  cudaError_t e = forward(n, B);
  const int BO = B * n->n_out;
  const int nb = blocks(BO);
  mse_kernel<<<nb, 256, 0, n->st>>>(n->y, t, n->dyb, n->dy, n->partial, BO, 1.f / (float)BO);
  if (e == cudaSuccess) e = backward(n, B);
  if (e == cudaSuccess && lr > 0.f) {
    ++n->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
    for (int i = 0; i < 6; ++i) {
      const int l = i / 2;
      const int cols = l == 0 ? n->n_in : n->width, ld = l == 0 ? n->ldx : cols;
      adam_kernel<<<blocks((long long)n->count[i]), 256, 0, n->st>>>(n->p[i], (i % 2 == 0) ? n->wb[l] : nullptr, cols, ld,
                                                                   n->g[i], n->m[i], n->v[i], (int)n->count[i], lr, b1,
                                                                   b2, c1, c2, 1e-8f);
    }
    refresh_wT(n);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && loss) {
    std::vector<double> part(nb);
    e = cudaMemcpyAsync(part.data(), n->partial, nb * sizeof(double), cudaMemcpyDeviceToHost, n->st);
    if (e == cudaSuccess) e = check_derr(n);
    double s = 0.0;
    for (double q : part) s += q;
    *loss = s / (double)BO;
  }
  return e == cudaSuccess ? SS_OK : mlp_fail(n, SS_ERR_CUDA, cudaGetErrorString(e));
}

int ss_mlp_use_tensor_cores(ss_mlp* n, int on) {
  if (!n) return SS_ERR_ARG;
  if (on && !n->w3T) return mlp_fail(n, SS_ERR_ARG, "tensor cores need width and n_out multiples of 8");
  if (on && !n->tc) {
    n->tc = 1;
    refresh_wT(n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mlp_fail(n, SS_ERR_CUDA, cudaGetErrorString(e));
  }
  n->tc = on ? 1 : 0;
  return SS_OK;
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
