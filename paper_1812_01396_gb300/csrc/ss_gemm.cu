// Batched complex128 GEMM on the FP64 pipe (sm_103a).
//
// Used for every product of the FP64 path: the Schur-complement update
// A_ii - A_{i,i+1} X_{i+1} and the chain Q_i = -X_i Q_{i-1} of Algorithm 1
// (Sec. 3B), the trailing updates of the blocked LU, the doubling products of
// the lead self-energies, the 2s x 2s boundary system R = 1 - C Q of Eq. x
// and the transmission products.
//
// Design: one launch covers a group of independent problems of any shapes.
// CTA b finds its problem by binary search in a prefix table of tile counts.
// Each CTA owns a TM x TN complex output tile (64 x 64, 16 x 256, 256 x 16,
// 16 x 64 or 64 x 16: per group the shape with the least padded work per busy
// SM, as the blocked LU's nb-deep updates are skinny and few),
// stages TM x 8 and 8 x TN slices of op(A) and op(B) in shared memory and
// keeps a 4 x 4 complex micro-tile per thread in registers.  On GB300 the FP64 pipe (about 2 DFMA per clock per SM) is the
// bound by a wide margin, so the kernel spends its effort on keeping every
// issued instruction a DFMA rather than on deep staging.
//
// Operands may be "formed": element = e*S - H read from two matrices, which
// fuses the assembly of A = E S - H into the loads (no A is ever stored).
#include "ss_internal.cuh"

namespace ss {

namespace {
constexpr int TK = 8, NT = 256;
// tile shapes by variant (TM x TN, micro-tile MI x MJ per thread):
//   0: 64 x 64 (4 x 4), 1: 16 x 256 (4 x 4), 2: 256 x 16 (4 x 4),
//   3: 16 x 64 (1 x 4), 4: 64 x 16 (4 x 1).
// The FP64 pipe, not shared memory, bounds every variant, so the small
// tiles only trade register reuse for more CTAs on small groups.
constexpr int NVAR = 5;
__host__ __device__ constexpr int tile_m(int v) { return v == 1 || v == 3 ? 16 : (v == 2 ? 256 : 64); }
__host__ __device__ constexpr int tile_n(int v) { return v == 1 ? 256 : (v == 2 || v == 4 ? 16 : 64); }
__host__ __device__ constexpr int micro_m(int v) { return v == 3 ? 1 : 4; }
__host__ __device__ constexpr int micro_n(int v) { return v == 4 ? 1 : 4; }

__device__ __forceinline__ int find_problem(const int* __restrict__ tile_start, int nprob, int bid) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(tile_start + mid) <= bid) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// element (i, j) of op(X)
__device__ __forceinline__ z64 op_load(const Operand& o, int i, int j) {
  size_t idx = o.trans ? (size_t)j * o.ld + i : (size_t)i * o.ld + j;
  z64 v = o.p[idx];
  if (o.s) {  // e S - H; real e (the device at real E) needs two FMAs, not a complex product
    const z64 sv = o.s[idx];
    v = o.e.y == 0.0 ? zmk(fma(o.e.x, sv.x, -v.x), fma(o.e.x, sv.y, -v.y)) : zsub(zmul(o.e, sv), v);
  }
  return o.trans ? zconj(v) : v;
}

template <typename R>
struct Cx;
template <>
struct Cx<double> {
  typedef double2 T;
  static __device__ __forceinline__ T cvt(z64 v) { return v; }
  static __device__ __forceinline__ z64 back(T v) { return v; }
};

// R = double: complex128 operands and accumulation (the only instance).
template <typename R, int V>
__global__ void __launch_bounds__(NT) zgemm_kernel(const GemmDesc* __restrict__ descs,
                                                   const int* __restrict__ tile_start, int nprob) {
  constexpr int TM = tile_m(V), TN = tile_n(V), MI = micro_m(V), MJ = micro_n(V);
  constexpr int TY = TM / MI, TX = TN / MJ;
  static_assert(TY * TX == NT, "one thread per micro-tile");
  typedef typename Cx<R>::T CT;
  __shared__ CT As[TK][TM];
  __shared__ CT Bs[TK][TN];
  const int pid = find_problem(tile_start, nprob, blockIdx.x);
  const GemmDesc& d = descs[pid];
  if (d.active && __ldg(d.active) == 0) return;
  const int m = d.m, n = d.n, K = d.k;
  const int tiles_n = (n + TN - 1) / TN;
  const int t = blockIdx.x - __ldg(tile_start + pid);
  const int row0 = (t / tiles_n) * TM, col0 = (t % tiles_n) * TN;
  if (d.lower && col0 >= row0 + TM) return;  // tile entirely above the diagonal
  const Operand a = d.a, b = d.b;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;

  CT acc[MI][MJ];
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < MJ; ++j) { acc[i][j].x = 0; acc[i][j].y = 0; }

  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = tid; e < TM * TK; e += NT) {
      int r, kk;
      if (a.trans) { kk = e / TM; r = e % TM; } else { r = e / TK; kk = e % TK; }
      const int gi = row0 + r, gk = k0 + kk;
      As[kk][r] = Cx<R>::cvt((gi < m && gk < K) ? op_load(a, gi, gk) : zmk(0.0, 0.0));
    }
    for (int e = tid; e < TK * TN; e += NT) {
      int c, kk;
      if (b.trans) { c = e / TK; kk = e % TK; } else { kk = e / TN; c = e % TN; }
      const int gj = col0 + c, gk = k0 + kk;
      Bs[kk][c] = Cx<R>::cvt((gj < n && gk < K) ? op_load(b, gk, gj) : zmk(0.0, 0.0));
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      CT av[MI], bv[MJ];
#pragma unroll
      for (int i = 0; i < MI; ++i) av[i] = As[kk][ty + TY * i];
#pragma unroll
      for (int j = 0; j < MJ; ++j) bv[j] = Bs[kk][tx + TX * j];
#pragma unroll
      for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < MJ; ++j) {
          acc[i][j].x = fma(av[i].x, bv[j].x, acc[i][j].x);
          acc[i][j].x = fma(-av[i].y, bv[j].y, acc[i][j].x);
          acc[i][j].y = fma(av[i].x, bv[j].y, acc[i][j].y);
          acc[i][j].y = fma(av[i].y, bv[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }

  const z64 alpha = d.alpha, beta = d.beta;
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
  // C - A B (the LU updates): no complex multiplies in the epilogue
  const bool sub = d.cmode == 0 && alpha.x == -1.0 && alpha.y == 0.0 && beta.x == 1.0 && beta.y == 0.0;
#pragma unroll
  for (int i = 0; i < MI; ++i) {
    const int r = row0 + ty + TY * i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < MJ; ++j) {
      const int c = col0 + tx + TX * j;
      if (c >= n) continue;
      if (sub) {
        const z64 p = Cx<R>::back(acc[i][j]);
        z64* cp = d.c + (size_t)r * d.ldc + c;
        const z64 o = *cp;
        *cp = zmk(o.x - p.x, o.y - p.y);
        continue;
      }
      z64 v = zmul(alpha, Cx<R>::back(acc[i][j]));
      if (d.cmode == 1) {
        const size_t fi = (size_t)r * d.ldcf + c;
        v = zadd(v, zmul(beta, zsub(zmul(d.ce, d.cs[fi]), d.ch[fi])));
      } else if (d.cmode == 2) {
        if (r == c) v = zadd(v, beta);
      } else if (use_beta) {
        v = zadd(v, zmul(beta, d.c[(size_t)r * d.ldc + c]));
      }
      d.c[(size_t)r * d.ldc + c] = v;
    }
  }
}
}  // namespace

int zgemm_tiles(int m, int n, int variant) {
  if (m <= 0 || n <= 0) return 0;
  const int tm = tile_m(variant), tn = tile_n(variant);
  return ((m + tm - 1) / tm) * ((n + tn - 1) / tn);
}

int zgemm_num_variants() { return NVAR; }

int zgemm_variant(const std::vector<GemmDesc>& ds) {
  // the tile shape with the least padded work per busy SM (ties: 64 x 64)
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 148;
  }
  double best = 0.0;
  int bv = 0;
  for (int v = 0; v < NVAR; ++v) {
    double work = 0.0, ctas = 0.0;
    for (auto& g : ds) {
      const int t = zgemm_tiles(g.m, g.n, v);
      work += (double)t * tile_m(v) * tile_n(v);
      ctas += t;
    }
    const double cost = work / std::min(ctas, (double)nsm);
    if (v == 0 || cost < best * 0.999) { best = cost; bv = v; }
  }
  return bv;
}

void launch_zgemm(const GemmDesc* d, const int* tile_start, int nprob, int total_tiles, cudaStream_t st,
                  int variant) {
  if (nprob <= 0 || total_tiles <= 0) return;
  switch (variant) {
    case 1: zgemm_kernel<double, 1><<<total_tiles, NT, 0, st>>>(d, tile_start, nprob); break;
    case 2: zgemm_kernel<double, 2><<<total_tiles, NT, 0, st>>>(d, tile_start, nprob); break;
    case 3: zgemm_kernel<double, 3><<<total_tiles, NT, 0, st>>>(d, tile_start, nprob); break;
    case 4: zgemm_kernel<double, 4><<<total_tiles, NT, 0, st>>>(d, tile_start, nprob); break;
    default: zgemm_kernel<double, 0><<<total_tiles, NT, 0, st>>>(d, tile_start, nprob);
  }
}

}  // namespace ss
