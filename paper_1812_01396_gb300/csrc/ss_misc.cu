// Elementwise forms, norms, traces and convergence flags (FP64).
//
//  zform   out = ax op(X) + ay op(Y) + az op(Z) + gamma I: builds A-blocks
//          E S - H at real E (Sec. 3B) or lead blocks z S - H at
//          z = E + i eta, right-hand sides, copies, Gamma = i(Sigma - Sigma^H).
//  norm1   max column sum of |a_ij| (the doubling's stopping test).
//  trace   sum_{a,b} A[a,b] B[b,a] = Tr[A B], the transmission reduction
//          (deterministic tree; one CTA per problem), or Tr[A] (density of
//          states).
#include "ss_internal.cuh"

namespace ss {

namespace {
constexpr int FT = 32;  // form tile edge
constexpr int FNT = 256;

__device__ __forceinline__ int find_problem(const int* __restrict__ tile_start, int nprob, int bid) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(tile_start + mid) <= bid) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// y + a x; a real coefficient (the common case) costs two FMAs on the slow
// FP64 pipe instead of a complex product and an add
__device__ __forceinline__ z64 zaxpy(z64 a, z64 x, z64 y) {
  if (a.y == 0.0) return zmk(fma(a.x, x.x, y.x), fma(a.x, x.y, y.y));
  return zadd(y, zmul(a, x));
}

__device__ __forceinline__ z64 opget(const z64* p, int ld, int tr, int r, int c) {
  return tr ? zconj(p[(size_t)c * ld + r]) : p[(size_t)r * ld + c];
}

__global__ void __launch_bounds__(FNT) zform_kernel(const FormDesc* __restrict__ descs,
                                                    const int* __restrict__ tile_start, int nprob) {
  const int pid = find_problem(tile_start, nprob, blockIdx.x);
  const FormDesc& d = descs[pid];
  if (d.active && __ldg(d.active) == 0) return;
  const int tiles_c = (d.cols + FT - 1) / FT;
  const int t = blockIdx.x - __ldg(tile_start + pid);
  const int r0 = (t / tiles_c) * FT, c0 = (t % tiles_c) * FT;
  // each thread handles 4 elements of the 32 x 32 tile
  const bool copy = d.x && !d.y && !d.z && !d.v && !d.nrm && d.ax.x == 1.0 && d.ax.y == 0.0 &&
                    d.gamma.x == 0.0 && d.gamma.y == 0.0;
  if (copy) {  // plain (conjugate-transposed) copy: no FP64 arithmetic, which is slow on this GPU
    for (int e = threadIdx.x; e < FT * FT; e += FNT) {
      const int r = r0 + e / FT, c = c0 + e % FT;
      if (r < d.rows && c < d.cols) d.out[(size_t)r * d.ldo + c] = opget(d.x, d.ldx, d.tx, r, c);
    }
    return;
  }
  double sq = 0.0;
  for (int e = threadIdx.x; e < FT * FT; e += FNT) {
    const int r = r0 + e / FT, c = c0 + e % FT;
    if (r >= d.rows || c >= d.cols) continue;
    z64 v = (r == c) ? d.gamma : zmk(0.0, 0.0);
    if (d.x) v = zaxpy(d.ax, opget(d.x, d.ldx, d.tx, r, c), v);
    if (d.y) v = zaxpy(d.ay, opget(d.y, d.ldy, d.ty, r, c), v);
    if (d.z) v = zaxpy(d.az, opget(d.z, d.ldz, d.tz, r, c), v);
    if (d.v) v = zaxpy(d.av, d.v[(size_t)r * d.ldv + c], v);
    if (d.nrm) sq = fma(v.x, v.x, fma(v.y, v.y, sq));
    else d.out[(size_t)r * d.ldo + c] = v;
  }
  if (d.nrm) {  // uniform per CTA
    __shared__ double red[FNT / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = 0.0;
      for (int q = 0; q < FNT / 32; ++q) b += red[q];
      atomicAdd(d.nrm, d.nw * b);
    }
  }
}

constexpr int RNT = 256;

// One thread per column, a CTA per 256 columns; the column sums are merged
// with an integer atomicMax on the IEEE bits (monotone for non-negative
// doubles; a NaN wins).  *out must be 0 before the launch.
__global__ void __launch_bounds__(RNT) norm1_kernel(const Norm1Desc* __restrict__ descs) {
  const Norm1Desc d = descs[blockIdx.y];
  if (d.active && __ldg(d.active) == 0) return;
  const int c = blockIdx.x * RNT + threadIdx.x;
  double sum = 0.0;
  if (c < d.cols) {
    for (int r = 0; r < d.rows; ++r) {
      const z64 v = d.a[(size_t)r * d.lda + c];
      sum += sqrt(fma(v.x, v.x, v.y * v.y));
    }
  }
  __shared__ double red[RNT / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_down_sync(0xffffffffu, sum, off);
    sum = (o > sum || o != o) ? o : sum;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = red[0];
    for (int q = 1; q < RNT / 32; ++q) b = (red[q] > b || red[q] != red[q]) ? red[q] : b;
    atomicMax(reinterpret_cast<unsigned long long*>(d.out),
              static_cast<unsigned long long>(__double_as_longlong(b)));
  }
}

__global__ void __launch_bounds__(RNT) trace_kernel(const TraceDesc* __restrict__ descs) {
  const TraceDesc d = descs[blockIdx.x];
  if (d.active && __ldg(d.active) == 0) return;
  // thread t sums rows a = t, t + RNT, ...; for each a it walks b.
  // b == nullptr: the trace of A itself (sum of its diagonal).
  z64 acc = zmk(0.0, 0.0);
  if (!d.b) {
    for (int a = threadIdx.x; a < d.n; a += RNT) acc = zadd(acc, d.a[(size_t)a * d.lda + a]);
  } else {
    for (int a = threadIdx.x; a < d.n; a += RNT) {
      for (int b = 0; b < d.n; ++b) {
        zfma(acc, d.a[(size_t)a * d.lda + b], d.b[(size_t)b * d.ldb + a]);
      }
    }
  }
  __shared__ z64 red[RNT / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    z64 s = red[0];
    for (int q = 1; q < RNT / 32; ++q) s = zadd(s, red[q]);
    *d.out = s;
  }
}

// After a doubling step (count = 1) or before the first one (count = 0):
// problems still active add `count` to their iteration counter, record
// convergence and drop out when converged, at the cap, or on a NaN norm.  The
// norms are reset to 0 for the next step's atomicMax.
__global__ void decim_check_kernel(double* __restrict__ na, double* __restrict__ nb,
                                   const double* __restrict__ nd, int* act, int* iters, int* conv,
                                   int nprob, double tol, int cap, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  const double a = na[p], b = nb[p];
  na[p] = 0.0;
  nb[p] = 0.0;
  if (!act[p]) return;
  iters[p] += count;
  const double m = fmax(a, b);
  const bool c = (m <= tol * nd[p]);
  conv[p] = c ? 1 : 0;
  if (c || iters[p] >= cap || m != m || a != a || b != b) act[p] = 0;
}
// sum |a_ij|^2 over an m x n block (one CTA per 256 columns, atomic add)
__global__ void __launch_bounds__(256) frob2_kernel(const Norm1Desc* __restrict__ descs) {
  const Norm1Desc d = descs[blockIdx.y];
  if (d.active && __ldg(d.active) == 0) return;
  const int c = blockIdx.x * 256 + threadIdx.x;
  double sum = 0.0;
  if (c < d.cols)
    for (int r = 0; r < d.rows; ++r) {
      const z64 v = d.a[(size_t)r * d.lda + c];
      sum = fma(v.x, v.x, fma(v.y, v.y, sum));
    }
  __shared__ double red[8];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int q = 0; q < 8; ++q) b += red[q];
    atomicAdd(d.out, b);
  }
}

// g (s x s complex, ld) = (y[0:s^2] + i y[s^2:2s^2]) * inv_scale, y fp32 row-major
__global__ void unpack_g_kernel(const float* __restrict__ y, int s, double inv_scale, z64* g, int ldg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s * s) return;
  const int r = i / s, c = i % s;
  g[(size_t)r * ldg + c] = zmk((double)y[i] * inv_scale, (double)y[(size_t)s * s + i] * inv_scale);
}

__global__ void real_part_kernel(const z64* __restrict__ in, double* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i].x;
}

__global__ void scaled_imag_kernel(const z64* __restrict__ in, double* __restrict__ out, int n, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = scale * in[i].y;
}

__global__ void fill_i32_kernel(int* p, int n, int v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
}  // namespace

void launch_frob2(const Norm1Desc* d, int nprob, int max_cols, cudaStream_t st) {
  if (nprob <= 0 || max_cols <= 0) return;
  dim3 grid((max_cols + 255) / 256, nprob);
  frob2_kernel<<<grid, 256, 0, st>>>(d);
}

void launch_unpack_g(const float* y, int s, double inv_scale, z64* g, int ldg, cudaStream_t st) {
  unpack_g_kernel<<<(s * s + 255) / 256, 256, 0, st>>>(y, s, inv_scale, g, ldg);
}

void launch_real_part(const z64* in, double* out, int n, cudaStream_t st) {
  if (n <= 0) return;
  real_part_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
}

void launch_scaled_imag(const z64* in, double* out, int n, double scale, cudaStream_t st) {
  if (n <= 0) return;
  scaled_imag_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, n, scale);
}

void launch_fill_i32(int* p, int n, int v, cudaStream_t st) {
  if (n <= 0) return;
  fill_i32_kernel<<<(n + 255) / 256, 256, 0, st>>>(p, n, v);
}

int zform_tiles(int rows, int cols) {
  if (rows <= 0 || cols <= 0) return 0;
  return ((rows + FT - 1) / FT) * ((cols + FT - 1) / FT);
}

void launch_zform(const FormDesc* d, const int* tile_start, int nprob, int total_tiles, cudaStream_t st) {
  if (nprob <= 0 || total_tiles <= 0) return;
  zform_kernel<<<total_tiles, FNT, 0, st>>>(d, tile_start, nprob);
}

void launch_norm1(const Norm1Desc* d, int nprob, int max_cols, cudaStream_t st) {
  if (nprob <= 0 || max_cols <= 0) return;
  dim3 grid((max_cols + RNT - 1) / RNT, nprob);
  norm1_kernel<<<grid, RNT, 0, st>>>(d);
}

void launch_trace(const TraceDesc* d, int nprob, cudaStream_t st) {
  if (nprob <= 0) return;
  trace_kernel<<<nprob, RNT, 0, st>>>(d);
}

void launch_decim_check(double* na, double* nb, const double* nd, int* act, int* iters, int* conv,
                        int nprob, double tol, int cap, int count, cudaStream_t st) {
  if (nprob <= 0) return;
  decim_check_kernel<<<(nprob + 127) / 128, 128, 0, st>>>(na, nb, nd, act, iters, conv, nprob, tol,
                                                          cap, count);
}

}  // namespace ss
