// Small dense complex eigenproblems K y = lambda y, one CTA per problem: the
// Rayleigh-Ritz step of the contour-integral (FEAST) lead solver (Sec. 3A,
// Eq. feast), whose reduced matrices have at most a few hundred rows.
//
// Standard algorithms, written from their definitions:
//   1. Householder reduction to upper Hessenberg form, H = Z^H K Z;
//   2. single-shift QR iteration on the Hessenberg matrix (implicit bulge
//      chase with Givens rotations, Wilkinson shift from the trailing 2 x 2
//      block, an exceptional shift every 10 steps without deflation),
//      accumulating Z, until H is upper triangular (the Schur form T);
//   3. eigenvectors of T by back substitution, x_j = 1, then y_j = Z x_j
//      (the caller multiplies by Z with its GEMM), normalised to unit norm.
// FP64 throughout; the matrices live in global memory (they stay in L1/L2),
// every rotation is applied by all threads of the CTA in parallel.  An
// iteration cap (30 steps per eigenvalue) sets *info = 1 instead of hanging.
#include "ss_internal.cuh"

namespace ss {

namespace {
constexpr int EIG_THREADS = 256;

__device__ __forceinline__ double zabs2(z64 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double zabs(z64 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ z64 zscale(z64 a, double s) { return zmk(a.x * s, a.y * s); }

// complex square root (principal branch)
__device__ __forceinline__ z64 zsqrt(z64 a) {
  const double r = zabs(a);
  if (r == 0.0) return zmk(0.0, 0.0);
  const double re = sqrt(0.5 * (r + fabs(a.x)));
  const double im = a.y / (2.0 * re);
  return a.x >= 0.0 ? zmk(re, im) : zmk(fabs(im), a.y >= 0.0 ? re : -re);
}

__global__ void __launch_bounds__(EIG_THREADS) eig_kernel(const EigDesc* __restrict__ descs) {
  const EigDesc d = descs[blockIdx.x];
  const int m = d.m;
  z64* __restrict__ H = d.h;  // m x m, ld = d.ld; overwritten by the Schur form
  z64* __restrict__ Z = d.z;  // m x m, ld = d.ld
  const int ld = d.ld;
  const int tid = threadIdx.x;
  __shared__ z64 v[512];
  __shared__ double rd[EIG_THREADS / 32];
  __shared__ z64 sh_c;
  __shared__ double sh_n;
  __shared__ int s_fail;
  if (tid == 0) s_fail = 0;
  // Z = 1
  for (int e = tid; e < m * m; e += EIG_THREADS) Z[(size_t)(e / m) * ld + e % m] = zmk((e / m) == (e % m) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  // ---- 1. Hessenberg reduction
  for (int k = 0; k + 2 < m; ++k) {
    const int n = m - k - 1;  // length of x = H[k+1.., k]
    double part = 0.0;
    for (int i = tid; i < n; i += EIG_THREADS) {
      const z64 x = H[(size_t)(k + 1 + i) * ld + k];
      v[i] = x;
      part += zabs2(x);
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) rd[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int q = 0; q < EIG_THREADS / 32; ++q) t += rd[q];
      const double nx = sqrt(t);
      const z64 x0 = v[0];
      const double a0 = zabs(x0);
      const z64 ph = a0 > 0.0 ? zscale(x0, 1.0 / a0) : zmk(1.0, 0.0);
      // v = x + ph ||x|| e1 (no cancellation), then H <- (1 - 2 v v^H / v^H v) H (...)
      v[0] = zadd(x0, zscale(ph, nx));
      const double vv = t - a0 * a0 + zabs2(v[0]);
      sh_n = (nx == 0.0 || vv == 0.0) ? 0.0 : 2.0 / vv;
    }
    __syncthreads();
    const double beta = sh_n;
    if (beta == 0.0) continue;
    // left: rows k+1.., every column j >= k: H[:, j] -= beta v (v^H H[:, j])
    for (int j = k + tid; j < m; j += EIG_THREADS) {
      z64 dot = zmk(0.0, 0.0);
      for (int i = 0; i < n; ++i) zfma(dot, zconj(v[i]), H[(size_t)(k + 1 + i) * ld + j]);
      dot = zscale(dot, beta);
      for (int i = 0; i < n; ++i) {
        z64& h = H[(size_t)(k + 1 + i) * ld + j];
        h = zsub(h, zmul(v[i], dot));
      }
    }
    __syncthreads();
    // right: every row r, columns k+1..: H[r, :] -= beta (H[r, :] v) v^H ; same for Z
    for (int r = tid; r < 2 * m; r += EIG_THREADS) {
      z64* row = r < m ? H + (size_t)r * ld : Z + (size_t)(r - m) * ld;
      z64 dot = zmk(0.0, 0.0);
      for (int i = 0; i < n; ++i) zfma(dot, row[k + 1 + i], v[i]);
      dot = zscale(dot, beta);
      for (int i = 0; i < n; ++i) row[k + 1 + i] = zsub(row[k + 1 + i], zmul(dot, zconj(v[i])));
    }
    __syncthreads();
    for (int i = k + 2 + tid; i < m; i += EIG_THREADS) H[(size_t)i * ld + k] = zmk(0.0, 0.0);
    __syncthreads();
  }
  // ---- 2. shifted QR iteration
  const double eps = 2.220446049250313e-16;
  int hi = m - 1, its = 0, total = 0;
  while (hi > 0) {
    // deflation point
    int l = hi;
    for (; l > 0; --l) {
      const double s = zabs(H[(size_t)(l - 1) * ld + l - 1]) + zabs(H[(size_t)l * ld + l]);
      if (zabs(H[(size_t)l * ld + l - 1]) <= eps * (s > 0.0 ? s : 1.0)) break;
    }
    __syncthreads();
    if (l == hi) {
      if (tid == 0 && hi > 0) H[(size_t)hi * ld + hi - 1] = zmk(0.0, 0.0);
      --hi;
      its = 0;
      __syncthreads();
      continue;
    }
    if (l > 0 && tid == 0) H[(size_t)l * ld + l - 1] = zmk(0.0, 0.0);
    if (++total > 30 * m) {
      if (tid == 0) s_fail = 1;
      break;
    }
    ++its;
    // Wilkinson shift: eigenvalue of the trailing 2 x 2 closer to H[hi][hi]
    z64 mu;
    {
      const z64 a = H[(size_t)(hi - 1) * ld + hi - 1], b = H[(size_t)(hi - 1) * ld + hi];
      const z64 c = H[(size_t)hi * ld + hi - 1], dd = H[(size_t)hi * ld + hi];
      if (its % 10 == 0) {
        mu = zadd(dd, zmk(zabs(c), 0.0));  // exceptional shift
      } else {
        const z64 tr2 = zscale(zadd(a, dd), 0.5);
        const z64 df = zscale(zsub(a, dd), 0.5);
        const z64 sq = zsqrt(zadd(zmul(df, df), zmul(b, c)));
        const z64 l1 = zadd(tr2, sq), l2 = zsub(tr2, sq);
        mu = zabs2(zsub(l1, dd)) < zabs2(zsub(l2, dd)) ? l1 : l2;
      }
    }
    __syncthreads();
    // implicit single-shift bulge chase on [l, hi]
    for (int k = l; k < hi; ++k) {
      if (tid == 0) {
        z64 x, y;
        if (k == l) {
          x = zsub(H[(size_t)l * ld + l], mu);
          y = H[(size_t)(l + 1) * ld + l];
        } else {
          x = H[(size_t)k * ld + k - 1];
          y = H[(size_t)(k + 1) * ld + k - 1];
        }
        const double ax = zabs(x), ay = zabs(y), r = hypot(ax, ay);
        double c;
        z64 sv;
        if (r == 0.0) { c = 1.0; sv = zmk(0.0, 0.0); }
        else if (ax == 0.0) { c = 0.0; sv = zscale(zconj(y), 1.0 / ay); }
        else { c = ax / r; sv = zscale(zmul(zscale(x, 1.0 / ax), zconj(y)), 1.0 / r); }
        sh_n = c;
        sh_c = sv;
      }
      __syncthreads();
      const double c = sh_n;
      const z64 sv = sh_c;
      // left: rows k, k+1, columns from (k == l ? l : k - 1) to m - 1 (the full Schur form)
      const int j0 = k == l ? l : k - 1;
      for (int j = j0 + tid; j < m; j += EIG_THREADS) {
        const z64 a = H[(size_t)k * ld + j], b = H[(size_t)(k + 1) * ld + j];
        H[(size_t)k * ld + j] = zadd(zscale(a, c), zmul(sv, b));
        H[(size_t)(k + 1) * ld + j] = zsub(zscale(b, c), zmul(zconj(sv), a));
      }
      __syncthreads();
      // right: columns k, k+1, rows 0..min(k+2, hi); and Z (every row)
      const int i1 = min(k + 2, hi);
      for (int r = tid; r <= i1 + m; r += EIG_THREADS) {
        z64* row;
        if (r <= i1) row = H + (size_t)r * ld;
        else row = Z + (size_t)(r - i1 - 1) * ld;
        if (r > i1 && r - i1 - 1 >= m) continue;
        const z64 a = row[k], b = row[k + 1];
        row[k] = zadd(zscale(a, c), zmul(zconj(sv), b));
        row[k + 1] = zsub(zscale(b, c), zmul(sv, a));
      }
      __syncthreads();
    }
  }
  __syncthreads();
  // ---- 3. eigenvectors of the triangular T into d.x (column j for eigenvalue T[j][j])
  const double tn = [&]() {
    double t = 0.0;
    for (int i = 0; i < m; ++i) t = fmax(t, zabs(H[(size_t)i * ld + i]));
    return t > 0.0 ? t : 1.0;
  }();
  for (int j = tid; j < m; j += EIG_THREADS) {
    const z64 lam = H[(size_t)j * ld + j];
    d.lam[j] = lam;
    z64* x = d.x;
    for (int i = m - 1; i > j; --i) x[(size_t)i * ld + j] = zmk(0.0, 0.0);
    x[(size_t)j * ld + j] = zmk(1.0, 0.0);
    for (int i = j - 1; i >= 0; --i) {
      z64 acc = zmk(0.0, 0.0);
      for (int k = i + 1; k <= j; ++k) zfma(acc, H[(size_t)i * ld + k], x[(size_t)k * ld + j]);
      z64 den = zsub(H[(size_t)i * ld + i], lam);
      if (zabs(den) < eps * tn) den = zmk(eps * tn, 0.0);
      x[(size_t)i * ld + j] = zmul(zmk(-acc.x, -acc.y), zinv(den));
    }
  }
  __syncthreads();
  if (tid == 0 && d.info) *d.info = s_fail;
}
}  // namespace

void launch_eig(const EigDesc* d, int nprob, cudaStream_t st) {
  if (nprob <= 0) return;
  eig_kernel<<<nprob, EIG_THREADS, 0, st>>>(d);
}

}  // namespace ss
