// Batched blocked LU with partial pivoting and fused right-hand-side solve.
//
// Each problem is a row-major s x ncols matrix W = [D | B]; the kernels
// factor P D = L U in place and overwrite B with D^-1 B.  This is the
// "one LU factorization and one backward substitution" per block of
// Algorithm 1 (Sec. 3B, Sec. 3C), with row pivoting added: the paper's
// zgesv_nopiv has none.  Pivot: largest |re| + |im| in the column, lowest row
// on ties (any stable order gives the same x).
//
// Per panel of nb <= 32 columns starting at k0 (right-looking):
//   lu_panel    rows k0..s-1 of the panel, on an 8-CTA cluster per problem
//               (one CTA per problem for panels taller than 1024 rows);
//   lu_rowblock applies the panel's row swaps to every other column and
//               forms U12 = L11^-1 A12 (and L11^-1 B1) in place;
//   (zgemm)     A22 -= L21 U12 over the trailing columns, RHS included.
// Two-level blocking (outer width nbo, a multiple of nb) keeps the nb-wide
// steps inside the outer block and defers the columns right of it: after the
// block, its rows are solved there panel by panel (lu_rowblock `far` plus
// FP64 updates inside the block) and the trailing matrix gets one update of
// depth nbo, which is what the exact tensor-core GEMM wants.
// After the last panel, B holds L^-1 P B; per panel from the bottom:
//   lu_backsub_diag  B_k = U_kk^-1 B_k,  (zgemm) B_0..k -= U_0..k,k B_k.
//
// A zero or non-finite pivot records 1 + its column in *info (first one
// only) and the elimination continues with a zero reciprocal, so no problem
// can stall the group.
#include <cooperative_groups.h>

#include "ss_internal.cuh"

namespace ss {

namespace {
constexpr int PANEL_THREADS = 512;
constexpr int NWARP = PANEL_THREADS / 32;
constexpr int MAXNB = 32;

__global__ void __launch_bounds__(PANEL_THREADS) lu_panel_kernel(const LuDesc* __restrict__ descs,
                                                                 int k0, int nb) {
  const LuDesc d = descs[blockIdx.x];
  if (d.active && __ldg(d.active) == 0) return;
  const int s = d.s;
  if (k0 >= s) return;
  const int nbw = min(nb, s - k0);
  z64* __restrict__ w = d.w;
  const size_t ld = d.ldw;
  __shared__ double red_v[NWARP];
  __shared__ int red_i[NWARP];
  __shared__ int red_bad[NWARP];
  __shared__ z64 prow[MAXNB];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int j = 0; j < nbw; ++j) {
    const int col = k0 + j;
    // --- pivot search over rows col..s-1
    double best = -1.0;
    int bi = s;
    int bad_elem = 0;
    for (int r = col + tid; r < s; r += PANEL_THREADS) {
      const z64 v = w[(size_t)r * ld + col];
      const double a = fabs(v.x) + fabs(v.y);
      if (!(a <= 1.7976931348623157e308)) bad_elem = 1;  // NaN or Inf in the column
      if (a > best) { best = a; bi = r; }
    }
    bad_elem = __any_sync(0xffffffffu, bad_elem);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; red_bad[warp] = bad_elem; }
    __syncthreads();
    if (tid == 0) {
      double bv = red_v[0];
      int bix = red_i[0];
      int anybad = red_bad[0];
      for (int q = 1; q < NWARP; ++q) {
        if (red_v[q] > bv || (red_v[q] == bv && red_i[q] < bix)) { bv = red_v[q]; bix = red_i[q]; }
        anybad |= red_bad[q];
      }
      const bool bad = anybad || !(bv > 0.0) || !isfinite(bv) || bix >= s;
      if (bix >= s) bix = col;
      if (bad && d.info && *d.info == 0) *d.info = col + 1;
      d.ipiv[col] = bix;
      s_piv = bix;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != col && tid < nbw) {
      z64* a = w + (size_t)col * ld + k0 + tid;
      z64* b = w + (size_t)p * ld + k0 + tid;
      const z64 t = *a;
      *a = *b;
      *b = t;
    }
    __syncthreads();
    if (tid < nbw) prow[tid] = w[(size_t)col * ld + k0 + tid];
    __syncthreads();
    const z64 inv = zinv(prow[j]);
    const z64 pr = (lane < nbw) ? prow[lane] : zmk(0.0, 0.0);
    // --- scale the column and update the rest of the panel, one row per warp
    for (int r = col + 1 + warp; r < s; r += NWARP) {
      z64* rowp = w + (size_t)r * ld + k0;
      const z64 l = zmul(rowp[j], inv);
      if (lane == j) rowp[j] = l;
      else if (lane > j && lane < nbw) rowp[lane] = zsub(rowp[lane], zmul(l, pr));
    }
    __syncthreads();
  }
}

// Register-resident panel: thread t keeps rows k0 + t + 512 q (q < RPT) of
// the panel, all NB columns, in registers for the whole factorisation; the
// pivot row and the row it replaces are exchanged through shared memory.
// Three barriers per column and no global traffic between load and store.
// Needs s - k0 <= 512 * RPT and NB * RPT <= 16 complex values per thread
// (64 registers of data).
// The column loop is a compile-time recursion so every register index is a
// constant.
struct PanelShared {
  double red_v[NWARP];
  int red_i[NWARP];
  int red_bad[NWARP];
  z64 prow[MAXNB];
  z64 crow[MAXNB];
  int piv;
};

template <int NB, int RPT, int J>
struct PanelStep {
  static __device__ __forceinline__ void run(z64 (&a)[RPT][NB], const int (&rows)[RPT], PanelShared& sh,
                                             const LuDesc& d, int k0, int nbw, int s) {
    if (J < nbw) {
      const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
      const int col = k0 + J;
      double best = -1.0;
      int bi = s, bad = 0;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        if (rows[q] >= col && rows[q] < s) {
          const double v = fabs(a[q][J].x) + fabs(a[q][J].y);
          if (!(v <= 1.7976931348623157e308)) bad = 1;
          if (v > best) { best = v; bi = rows[q]; }
        }
      }
      bad = __any_sync(0xffffffffu, bad);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) { sh.red_v[warp] = best; sh.red_i[warp] = bi; sh.red_bad[warp] = bad; }
      __syncthreads();
      if (tid == 0) {
        double bv = sh.red_v[0];
        int bix = sh.red_i[0], anybad = sh.red_bad[0];
        for (int q = 1; q < NWARP; ++q) {
          if (sh.red_v[q] > bv || (sh.red_v[q] == bv && sh.red_i[q] < bix)) { bv = sh.red_v[q]; bix = sh.red_i[q]; }
          anybad |= sh.red_bad[q];
        }
        const bool badp = anybad || !(bv > 0.0) || !isfinite(bv) || bix >= s;
        if (bix >= s) bix = col;
        if (badp && d.info && *d.info == 0) *d.info = col + 1;
        d.ipiv[col] = bix;
        sh.piv = bix;
      }
      __syncthreads();
      const int p = sh.piv;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        if (rows[q] == p) {
#pragma unroll
          for (int c = 0; c < NB; ++c) sh.prow[c] = a[q][c];
        }
        if (rows[q] == col && p != col) {
#pragma unroll
          for (int c = 0; c < NB; ++c) sh.crow[c] = a[q][c];
        }
      }
      __syncthreads();
      if (p != col) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          if (rows[q] == col) {
#pragma unroll
            for (int c = 0; c < NB; ++c) a[q][c] = sh.prow[c];
          } else if (rows[q] == p) {
#pragma unroll
            for (int c = 0; c < NB; ++c) a[q][c] = sh.crow[c];
          }
        }
      }
      const z64 inv = zinv(sh.prow[J]);
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        if (rows[q] > col && rows[q] < s) {
          const z64 l = zmul(a[q][J], inv);
          a[q][J] = l;
#pragma unroll
          for (int c = J + 1; c < NB; ++c) {
            const z64 u = sh.prow[c];
            a[q][c].x = fma(-l.x, u.x, a[q][c].x);
            a[q][c].x = fma(l.y, u.y, a[q][c].x);
            a[q][c].y = fma(-l.x, u.y, a[q][c].y);
            a[q][c].y = fma(-l.y, u.x, a[q][c].y);
          }
        }
      }
    }
    PanelStep<NB, RPT, J + 1>::run(a, rows, sh, d, k0, nbw, s);
  }
};

template <int NB, int RPT>
struct PanelStep<NB, RPT, NB> {
  static __device__ __forceinline__ void run(z64 (&)[RPT][NB], const int (&)[RPT], PanelShared&, const LuDesc&,
                                             int, int, int) {}
};

template <int NB, int RPT>
__global__ void __launch_bounds__(PANEL_THREADS, 1) lu_panel_reg_kernel(const LuDesc* __restrict__ descs,
                                                                     int k0, int nb) {
  const LuDesc d = descs[blockIdx.x];
  if (d.active && __ldg(d.active) == 0) return;
  const int s = d.s;
  if (k0 >= s) return;
  const int nbw = min(min(nb, NB), s - k0);
  z64* __restrict__ w = d.w;
  const size_t ld = d.ldw;
  __shared__ PanelShared sh;
  z64 a[RPT][NB];
  int rows[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    rows[q] = k0 + threadIdx.x + q * PANEL_THREADS;
#pragma unroll
    for (int c = 0; c < NB; ++c)
      a[q][c] = (rows[q] < s && c < nbw) ? w[(size_t)rows[q] * ld + k0 + c] : zmk(0.0, 0.0);
  }
  PanelStep<NB, RPT, 0>::run(a, rows, sh, d, k0, nbw, s);
#pragma unroll
  for (int q = 0; q < RPT; ++q)
    if (rows[q] < s) {
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < nbw) w[(size_t)rows[q] * ld + k0 + c] = a[q][c];
    }
}

// Cluster panel: the panel of one problem is spread over a cluster of CL
// CTAs (CL SMs), because a single SM retires only about two FP64 FMAs per
// clock.  Row k0 + c + CL t lives in thread t of cluster rank c, in
// registers.  Per column one cluster barrier: before it every CTA publishes
// its local pivot candidate (modulus, row, the row's values) and the owner of
// the diagonal row publishes that row, all in its own shared memory; after it
// every CTA reads the CL candidates through distributed shared memory, picks
// the same pivot (largest |re| + |im|, lowest row on ties) and swaps and
// updates its own rows.  The published slots alternate between two buffers,
// so a slot is rewritten only after every CTA has passed the next barrier.
// Same arithmetic, in the same order, as the single-CTA kernels.
template <int NB, int CL>
struct ClusterPanelShared {
  // published for the other CTAs of the cluster (two buffers)
  double cval[2];
  int cidx[2], cbad[2];
  z64 cand_row[2][NB];
  z64 diag_row[2][NB];
  // this CTA's copies of every CTA's candidate and of the diagonal row
  double rval[CL];
  int ridx[CL], rbad[CL];
  z64 rrow[CL][NB];
  z64 crow[NB];
  double wv[4];
  int wi[4], wb[4];
  int piv, win;
  z64 inv;
};

template <int NB, int CL, int NT>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT) lu_panel_cluster_kernel(
    const LuDesc* __restrict__ descs, int k0, int nb) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const LuDesc d = descs[blockIdx.x / CL];
  __shared__ ClusterPanelShared<NB, CL> sh;
  const bool live = !(d.active && __ldg(d.active) == 0) && k0 < d.s;  // same for the whole cluster
  if (live) {
    const int s = d.s;
    const int nbw = min(min(nb, NB), s - k0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row = k0 + crank + CL * tid;
    z64* __restrict__ w = d.w;
    const size_t ld = d.ldw;
    z64 a[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) a[c] = (row < s && c < nbw) ? w[(size_t)row * ld + k0 + c] : zmk(0.0, 0.0);
#pragma unroll
    for (int J = 0; J < NB; ++J) {
      if (J < nbw) {
        const int col = k0 + J, buf = J & 1;
        // local candidate
        double best = -1.0;
        int bi = s, bad = 0;
        if (row >= col && row < s) {
          const double v = fabs(a[J].x) + fabs(a[J].y);
          if (!(v <= 1.7976931348623157e308)) bad = 1;
          if (v > best) { best = v; bi = row; }
        }
        bad = __any_sync(0xffffffffu, bad);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const double ov = __shfl_down_sync(0xffffffffu, best, off);
          const int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { sh.wv[warp] = best; sh.wi[warp] = bi; sh.wb[warp] = bad; }
        __syncthreads();
        // every thread reduces the warp results, so the CTA's winner knows itself
        double cbv = sh.wv[0];
        int cbix = sh.wi[0], canyb = sh.wb[0];
#pragma unroll
        for (int q = 1; q < NT / 32; ++q) {
          if (sh.wv[q] > cbv || (sh.wv[q] == cbv && sh.wi[q] < cbix)) { cbv = sh.wv[q]; cbix = sh.wi[q]; }
          canyb |= sh.wb[q];
        }
        if (tid == 0) { sh.cval[buf] = cbv; sh.cidx[buf] = cbix; sh.cbad[buf] = canyb; }
        if (row < s && row == cbix) {
#pragma unroll
          for (int c = 0; c < NB; ++c) sh.cand_row[buf][c] = a[c];
        }
        if (row == col) {
#pragma unroll
          for (int c = 0; c < NB; ++c) sh.diag_row[buf][c] = a[c];
        }
        cluster.sync();
        // one round of distributed shared memory reads: every CTA's candidate
        // (modulus, row index, values) and the diagonal row
        {
          constexpr int NR = CL * (NB + 1) + NB, NI = (NR + NT - 1) / NT;
          const int cc = (col - k0) % CL;
          z64 vals[NI];
#pragma unroll
          for (int i = 0; i < NI; ++i) {
            const int e = tid + i * NT;
            vals[i] = zmk(0.0, 0.0);
            if (e < CL) {
              const ClusterPanelShared<NB, CL>* o = cluster.map_shared_rank(&sh, e);
              vals[i] = zmk(o->cval[buf], __hiloint2double(o->cbad[buf], o->cidx[buf]));
            } else if (e < CL + CL * NB) {
              const int q = (e - CL) / NB, c = (e - CL) % NB;
              vals[i] = cluster.map_shared_rank(&sh, q)->cand_row[buf][c];
            } else if (e < NR) {
              vals[i] = cluster.map_shared_rank(&sh, cc)->diag_row[buf][e - CL - CL * NB];
            }
          }
#pragma unroll
          for (int i = 0; i < NI; ++i) {
            const int e = tid + i * NT;
            if (e < CL) {
              sh.rval[e] = vals[i].x;
              sh.ridx[e] = __double2loint(vals[i].y);
              sh.rbad[e] = __double2hiint(vals[i].y);
            } else if (e < CL + CL * NB) {
              sh.rrow[(e - CL) / NB][(e - CL) % NB] = vals[i];
            } else if (e < NR) {
              sh.crow[e - CL - CL * NB] = vals[i];
            }
          }
        }
        __syncthreads();
        // global pivot (largest modulus, lowest row on ties), its reciprocal
        if (tid == 0) {
          double bv = sh.rval[0];
          int bix = sh.ridx[0], anyb = sh.rbad[0], win = 0;
          for (int q = 1; q < CL; ++q) {
            if (sh.rval[q] > bv || (sh.rval[q] == bv && sh.ridx[q] < bix)) { bv = sh.rval[q]; bix = sh.ridx[q]; win = q; }
            anyb |= sh.rbad[q];
          }
          const bool badp = anyb || !(bv > 0.0) || !isfinite(bv) || bix >= s;
          if (bix >= s) bix = col;
          // the winner's published candidate row is the pivot row (the
          // diagonal row itself when it wins or the column has no usable entry)
          sh.piv = bix;
          sh.win = (bix == col) ? -1 : win;
          sh.inv = zinv(bix == col ? sh.crow[J] : sh.rrow[win][J]);
          if (crank == 0) {
            if (badp && d.info && *d.info == 0) *d.info = col + 1;
            d.ipiv[col] = bix;
          }
        }
        __syncthreads();
        const z64* prow = sh.win < 0 ? sh.crow : sh.rrow[sh.win];
        const int p = sh.piv;
        if (p != col) {
          if (row == col) {
#pragma unroll
            for (int c = 0; c < NB; ++c) a[c] = prow[c];
          } else if (row == p) {
#pragma unroll
            for (int c = 0; c < NB; ++c) a[c] = sh.crow[c];
          }
        }
        if (row > col && row < s) {
          const z64 l = zmul(a[J], sh.inv);
          a[J] = l;
#pragma unroll
          for (int c = J + 1; c < NB; ++c) {
            const z64 u = prow[c];
            a[c].x = fma(-l.x, u.x, a[c].x);
            a[c].x = fma(l.y, u.y, a[c].x);
            a[c].y = fma(-l.x, u.y, a[c].y);
            a[c].y = fma(-l.y, u.x, a[c].y);
          }
        }
      }
    }
    if (row < s) {
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < nbw) w[(size_t)row * ld + k0 + c] = a[c];
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// Tournament pivoting panel (a communication-avoiding LU of the tall panel).
// Rows are spread over an 8-CTA cluster as in lu_panel_cluster_kernel
// (row k0 + c + CL t in thread t of cluster rank c):
//   1. every CTA runs partial pivoting on its own rows only (CTA-local
//      barriers) and offers the rows it picked, with their original values,
//      as candidates; the owners of rows k0..k0+NB-1 publish those rows too;
//   2. one cluster barrier; every CTA reads the CL x NB candidates through
//      distributed shared memory and runs the same partial pivoting on them
//      (largest |re| + |im|, lowest row on ties): that selects the NB pivot
//      rows in order and yields the factored pivot block [L11 \ U11], the same
//      in every CTA;
//   3. the pivot rows applied as NB successive row exchanges (recorded in
//      ipiv, as partial pivoting does) tell each thread which original row
//      ends up in its position; that row times U11^-1 is its row of L21.
// Two cluster barriers per panel instead of one per column.  The pivots may
// differ from partial pivoting's (another stable choice); the result is an
// exact P A = L U of the panel in the LU code's layout.
template <int NB, int CL, int NT>
struct TsluShared {
  z64 pubC[NB][NB];   // this CTA's candidates (original rows), published
  int pubId[NB];
  int pubN;
  z64 pubT[NB][NB];   // original rows k0 + i owned by this CTA, published
  z64 C[CL * NB][NB]; // gathered candidates, then their elimination
  int cid[CL * NB];
  int nc;
  int cbase[CL];      // first slot of each CTA's candidates
  z64 T[NB][NB];      // rows k0 .. k0 + NB - 1, original
  z64 prow[NB];
  double wv[NT / 32];
  int wi[NT / 32];
  int win, bad;
  int ipv[NB];
  int pivc[NB];       // candidate slot of pivot j
};

template <int NB, int NT>
__device__ __forceinline__ void cta_argmax(double v, int idx, double (&wv)[NT / 32], int (&wi)[NT / 32], int& out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, off);
    const int oi = __shfl_down_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if (lane == 0) { wv[warp] = v; wi[warp] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = wv[0];
    int bi = wi[0];
    for (int q = 1; q < NT / 32; ++q)
      if (wv[q] > bv || (wv[q] == bv && wi[q] < bi)) { bv = wv[q]; bi = wi[q]; }
    out = bv >= 0.0 ? bi : -1;
  }
  __syncthreads();
}

template <int NB, int CL, int NT>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT) lu_panel_tslu_kernel(
    const LuDesc* __restrict__ descs, int k0, int nb) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const LuDesc d = descs[blockIdx.x / CL];
  __shared__ TsluShared<NB, CL, NT> sh;
  const bool live = !(d.active && __ldg(d.active) == 0) && k0 < d.s;  // same for the whole cluster
  const int tid = threadIdx.x;
  const int s = d.s;
  const int nbw = live ? min(min(nb, NB), s - k0) : 0;
  const int row = k0 + crank + CL * tid;
  const bool valid = live && row < s;
  z64* __restrict__ w = d.w;
  const size_t ld = d.ldw;
  z64 a[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) a[c] = (valid && c < nbw) ? w[(size_t)row * ld + k0 + c] : zmk(0.0, 0.0);
  if (tid == 0) sh.pubN = 0;
  // ---- 1. local partial pivoting on this CTA's rows: candidates
  {
    z64 b[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) b[c] = a[c];
    bool chosen = false;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j < nbw) {  // nbw is uniform over the CTA
        const double v = (valid && !chosen) ? fabs(b[j].x) + fabs(b[j].y) : -1.0;
        const double vv = (v == v) ? v : 1.7976931348623157e308;  // NaN rows first (reported below)
        cta_argmax<NB, NT>(vv, valid ? row : s + CL * NT, sh.wv, sh.wi, sh.win);
        const int wrow = sh.win;
        if (wrow >= 0) {
          if (row == wrow) {
            chosen = true;
#pragma unroll
            for (int c = 0; c < NB; ++c) { sh.prow[c] = b[c]; sh.pubC[j][c] = a[c]; }
            sh.pubId[j] = row;
            sh.pubN = j + 1;
          }
          __syncthreads();
          if (valid && !chosen) {
            const z64 p = sh.prow[j];
            const z64 l = zmul(b[j], zinv(p));
#pragma unroll
            for (int c = j + 1; c < NB; ++c) {
              const z64 u = sh.prow[c];
              b[c].x = fma(-l.x, u.x, b[c].x);
              b[c].x = fma(l.y, u.y, b[c].x);
              b[c].y = fma(-l.x, u.y, b[c].y);
              b[c].y = fma(-l.y, u.x, b[c].y);
            }
          }
        }
        __syncthreads();
      }
    }
  }
  if (valid && row < k0 + nbw) {
#pragma unroll
    for (int c = 0; c < NB; ++c) sh.pubT[row - k0][c] = a[c];
  }
  cluster.sync();
  // ---- 2. gather every CTA's candidates and the top rows; partial pivoting on them
  if (nbw > 0) {
    if (tid == 0) {
      int n = 0;
      for (int q = 0; q < CL; ++q) {
        const TsluShared<NB, CL, NT>* o = cluster.map_shared_rank(&sh, q);
        const int m = o->pubN;
        sh.cbase[q] = n;
        for (int i = 0; i < m; ++i) sh.cid[n + i] = o->pubId[i];
        n += m;
      }
      sh.nc = n;
    }
    __syncthreads();
    // values: candidate slot cbase[q] + i holds CTA q's i-th candidate
    for (int e = tid; e < CL * NB * NB; e += NT) {
      const int q = e / (NB * NB), i = (e / NB) % NB, c = e % NB;
      const int m = (q + 1 < CL ? sh.cbase[q + 1] : sh.nc) - sh.cbase[q];
      if (i < m) sh.C[sh.cbase[q] + i][c] = cluster.map_shared_rank(&sh, q)->pubC[i][c];
    }
    for (int e = tid; e < nbw * NB; e += NT) {
      const int i = e / NB, c = e % NB;
      sh.T[i][c] = cluster.map_shared_rank(&sh, i % CL)->pubT[i][c];
    }
    if (tid == 0) sh.bad = 0;
    __syncthreads();
    const int nc = sh.nc;
    // candidate slots handled by this thread: tid, tid + NT (nc <= CL * NB <= 2 NT)
    bool ch0 = false, ch1 = false;
    for (int j = 0; j < nbw; ++j) {
      double v = -1.0;
      int vi = s + CL * NT;
      int slot = -1;
      for (int h = 0; h < 2; ++h) {
        const int e = tid + h * NT;
        if (e < nc && !(h ? ch1 : ch0)) {
          const z64 x = sh.C[e][j];
          double a1 = fabs(x.x) + fabs(x.y);
          if (!(a1 == a1)) a1 = 1.7976931348623157e308;
          if (a1 > v || (a1 == v && sh.cid[e] < vi)) { v = a1; vi = sh.cid[e]; slot = e; }
        }
      }
      // argmax over (value, original row); the slot travels with the row index
      cta_argmax<NB, NT>(v, vi, sh.wv, sh.wi, sh.win);
      const int wrow = sh.win;
      if (slot >= 0 && sh.cid[slot] == wrow) {
        sh.pivc[j] = slot;
        if (slot == tid) ch0 = true; else ch1 = true;
        const z64 pv = sh.C[slot][j];
        const double ap = fabs(pv.x) + fabs(pv.y);
        if (!(ap > 0.0 && ap <= 1.7976931348623157e308) && sh.bad == 0) sh.bad = j + 1;
      }
      __syncthreads();
      const int ps = sh.pivc[j];
      const z64 inv = zinv(sh.C[ps][j]);
      for (int h = 0; h < 2; ++h) {
        const int e = tid + h * NT;
        if (e < nc && !(h ? ch1 : ch0)) {
          const z64 l = zmul(sh.C[e][j], inv);
          sh.C[e][j] = l;  // multiplier (kept for the pivot block rows)
          for (int c = j + 1; c < NB; ++c) sh.C[e][c] = zsub(sh.C[e][c], zmul(l, sh.C[ps][c]));
        }
      }
      __syncthreads();
    }
    // pivot rows as successive exchanges (row positions), one thread
    if (tid == 0) {
      int pos_row[2 * NB], pos_at[2 * NB], np = 0;  // (position -> row) for touched positions
      for (int j = 0; j < nbw; ++j) {
        const int prw = sh.cid[sh.pivc[j]];
        // current position of row prw
        int p = prw;
        for (int t = 0; t < np; ++t)
          if (pos_row[t] == prw) { p = pos_at[t]; break; }
        sh.ipv[j] = p;
        // swap the contents of positions k0 + j and p
        const int a1 = k0 + j;
        int r1 = a1, r2 = p;  // rows currently at a1 and p
        int t1 = -1, t2 = -1;
        for (int t = 0; t < np; ++t) { if (pos_at[t] == a1) t1 = t; if (pos_at[t] == p) t2 = t; }
        if (t1 >= 0) r1 = pos_row[t1];
        if (t2 >= 0) r2 = pos_row[t2];
        if (t1 < 0) { t1 = np; pos_at[np] = a1; ++np; }
        if (t2 < 0 && p != a1) { t2 = np; pos_at[np] = p; ++np; }
        pos_row[t1] = r2;
        if (p != a1) pos_row[t2] = r1;
      }
      if (crank == 0) {
        for (int j = 0; j < nbw; ++j) d.ipiv[k0 + j] = sh.ipv[j];
        if (sh.bad && d.info && *d.info == 0) *d.info = k0 + sh.bad;
      }
    }
    __syncthreads();
    // ---- 3. this thread's final row
    if (valid) {
      if (row < k0 + nbw) {
        const int ps = sh.pivc[row - k0];
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c < nbw) w[(size_t)row * ld + k0 + c] = sh.C[ps][c];
      } else {
        int src = row;
        for (int j = nbw - 1; j >= 0; --j) {
          if (src == k0 + j) src = sh.ipv[j];
          else if (src == sh.ipv[j]) src = k0 + j;
        }
        // a row moved below the pivot block always comes from the block's original rows
        const bool from_top = src != row && src >= k0 && src < k0 + nbw;
        z64 x[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) x[c] = from_top ? sh.T[src - k0][c] : a[c];
        // L row = x U11^-1, U11 = upper part of the pivot block
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          if (j < nbw) {
            z64 acc = x[j];
#pragma unroll
            for (int c = 0; c < j; ++c) {
              const z64 u = sh.C[sh.pivc[c]][j];
              acc.x = fma(-x[c].x, u.x, acc.x);
              acc.x = fma(x[c].y, u.y, acc.x);
              acc.y = fma(-x[c].x, u.y, acc.y);
              acc.y = fma(-x[c].y, u.x, acc.y);
            }
            x[j] = zmul(acc, zinv(sh.C[sh.pivc[j]][j]));
          }
        }
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c < nbw) w[(size_t)row * ld + k0 + c] = x[c];
      }
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

constexpr int RB_THREADS = 64;  // one thread per column; small CTAs spread the FP64 work over more SMs

// Row swaps on every column outside the panel, then U12 = L11^-1 A12 on the
// columns to its right (right-hand sides included).  With an outer block
// width nbo > 0 (two-level blocking) the solve stops at the end of the outer
// block, K1 = min(K0 + nbo, s): columns from K1 on are swapped now and solved
// later by the `far` variant, which applies no swaps and solves the rows of
// this panel on columns K1..ncols-1 only.  The L factors left of the outer
// block are never read again (only the right-hand sides are), so their rows
// are left unswapped.  One thread per column; NB >= nb is
// the compile-time panel width, and each dot product runs in two halves
// (even / odd terms) to shorten the dependent FMA chains.
template <int NB>
__global__ void __launch_bounds__(RB_THREADS) lu_rowblock_kernel(const LuDesc* __restrict__ descs,
                                                                 int k0, int nb, int nbo, int far) {
  const LuDesc d = descs[blockIdx.y];
  if (d.active && __ldg(d.active) == 0) return;
  const int s = d.s;
  if (k0 >= s) return;
  const int nbw = min(min(nb, NB), s - k0);
  // nbo < 0 (Hermitian factorisation): only the right-hand-side columns, from s on
  const int K1 = nbo > 0 ? min((k0 / nbo) * nbo + nbo, s) : (nbo < 0 ? s : d.ncols);
  __shared__ z64 Ls[NB][NB + 1];
  __shared__ int piv[NB];
  for (int e = threadIdx.x; e < nbw * nbw; e += RB_THREADS) {
    const int r = e / nbw, c = e % nbw;
    Ls[r][c] = d.w[(size_t)(k0 + r) * d.ldw + k0 + c];
  }
  if (threadIdx.x < nbw) piv[threadIdx.x] = d.ipiv[k0 + threadIdx.x];
  __syncthreads();
  const int q = blockIdx.x * RB_THREADS + threadIdx.x;
  z64* __restrict__ w = d.w;
  const size_t ld = d.ldw;
  // far 0: row exchanges on every column from the outer block on, L11^-1 on the
  //        block's columns right of the panel;
  // far 1: L11^-1 on the columns right of the outer block (exchanged before);
  // far 2: as 0 with the exchanges limited to the outer block's columns;
  // far 3: the row exchanges of every panel of the outer block, in order, on
  //        the columns right of it, and nothing else (2 for each panel, then 3
  //        once, then 1 for each panel: the same operations in the same order
  //        on every column as 0 then 1, with the columns right of the block
  //        untouched until its far phase)
  auto exchange = [&](int c) {
    for (int j = 0; j < nbw; ++j) {
      const int p = piv[j];
      if (p != k0 + j) {
        z64* a = w + (size_t)(k0 + j) * ld + c;
        z64* b = w + (size_t)p * ld + c;
        const z64 t = *a;
        *a = *b;
        *b = t;
      }
    }
  };
  int c;
  if (far == 3) {
    if (nbo <= 0 || q >= d.ncols - K1) return;
    c = K1 + q;
    for (int r = (k0 / nbo) * nbo; r < K1; ++r) {
      const int p = d.ipiv[r];
      if (p != r) {
        z64* a = w + (size_t)r * ld + c;
        z64* b = w + (size_t)p * ld + c;
        const z64 t = *a;
        *a = *b;
        *b = t;
      }
    }
    return;
  }
  if (far == 1) {
    if (q >= d.ncols - K1) return;
    c = K1 + q;
  } else {
    // columns left of the outer block (left of the panel with one level)
    // hold L factors nothing reads again: they are not exchanged
    const int c0 = nbo > 0 ? (k0 / nbo) * nbo : k0;
    const int nout = (far == 2 ? K1 : d.ncols) - nbw - c0;
    if (q >= nout) return;
    c = (c0 + q < k0) ? c0 + q : c0 + q + nbw;
    exchange(c);
    if (c < k0 || c >= K1) return;
  }
  z64 x[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nbw) x[j] = w[(size_t)(k0 + j) * ld + c];
#pragma unroll
  for (int j = 1; j < NB; ++j) {
    if (j < nbw) {
      z64 e0 = x[j], e1 = zmk(0.0, 0.0);
#pragma unroll
      for (int i = 0; i < j; ++i) {
        const z64 l = Ls[j][i];
        z64& acc = (i & 1) ? e1 : e0;
        acc.x = fma(-l.x, x[i].x, acc.x);
        acc.x = fma(l.y, x[i].y, acc.x);
        acc.y = fma(-l.x, x[i].y, acc.y);
        acc.y = fma(-l.y, x[i].x, acc.y);
      }
      x[j] = zadd(e0, e1);
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nbw) w[(size_t)(k0 + j) * ld + c] = x[j];
}

// Every row exchange of the outer block [K0, K1) (pivots ipiv[K0 .. K1-1],
// applied in order) on the columns right of it, as one permutation: thread 0
// composes the exchanges on a map of rows K0 .. s-1 in shared memory and lists
// the rows whose values move (at most 2 (K1 - K0)); then XC columns per CTA
// read every moving row's source value and, after a barrier, write it to its
// destination.  The same data movement as the exchanges one after the other,
// with no chain of dependent loads.
constexpr int XC = 8, XT = 256;
constexpr size_t XSMEM_MAX = 96 * 1024;
size_t exchange_smem(int max_rows, int nbo) {
  return (size_t)max_rows * 4 + (size_t)4 * nbo * 4 + 16 + (size_t)2 * nbo * XC * sizeof(z64);
}

__global__ void __launch_bounds__(XT) lu_block_exchange_kernel(const LuDesc* __restrict__ descs, int K0, int nbo) {
  const LuDesc d = descs[blockIdx.y];
  if (d.active && __ldg(d.active) == 0) return;
  const int s = d.s;
  if (K0 >= s) return;
  const int K1 = min(K0 + nbo, s);
  const int cbase = K1 + blockIdx.x * XC;
  if (cbase >= d.ncols) return;
  extern __shared__ __align__(16) unsigned char xsm[];
  int* map = reinterpret_cast<int*>(xsm);  // row K0 + i receives the values of row map[i]
  int* dst = map + (s - K0);
  int* src = dst + 2 * nbo;
  z64* stage = reinterpret_cast<z64*>((reinterpret_cast<uintptr_t>(src + 2 * nbo) + 15) & ~uintptr_t(15));
  __shared__ int naff;
  for (int i = threadIdx.x; i < s - K0; i += XT) map[i] = K0 + i;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int r = K0; r < K1; ++r) {
      const int p = d.ipiv[r];
      if (p != r && p > r && p < s) {
        const int t = map[r - K0];
        map[r - K0] = map[p - K0];
        map[p - K0] = t;
      }
    }
    int n = 0;
    for (int r = K0; r < K1; ++r) {
      if (map[r - K0] != r) { dst[n] = r; src[n] = map[r - K0]; ++n; }
    }
    for (int r = K0; r < K1; ++r) {
      const int p = d.ipiv[r];
      if (p >= K1 && p < s && map[p - K0] != p) {  // listed once: its entry is reset below
        dst[n] = p;
        src[n] = map[p - K0];
        map[p - K0] = p;
        ++n;
      }
    }
    naff = n;
  }
  __syncthreads();
  const int n = naff;
  z64* __restrict__ w = d.w;
  const size_t ld = d.ldw;
  for (int e = threadIdx.x; e < n * XC; e += XT) {
    const int c = cbase + e % XC;
    if (c < d.ncols) stage[e] = w[(size_t)src[e / XC] * ld + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * XC; e += XT) {
    const int c = cbase + e % XC;
    if (c < d.ncols) w[(size_t)dst[e / XC] * ld + c] = stage[e];
  }
}

// B_k = U_kk^-1 B_k on the right-hand-side columns (backward substitution
// within one diagonal block of U), two FMA chains per dot product as above.
template <int NB>
__global__ void __launch_bounds__(RB_THREADS) lu_backsub_diag_kernel(const LuDesc* __restrict__ descs,
                                                                     int k0, int nb) {
  const LuDesc d = descs[blockIdx.y];
  if (d.active && __ldg(d.active) == 0) return;
  const int s = d.s;
  if (k0 >= s) return;
  const int nbw = min(min(nb, NB), s - k0);
  __shared__ z64 Us[NB][NB + 1];
  __shared__ z64 dinv[NB];
  for (int e = threadIdx.x; e < nbw * nbw; e += RB_THREADS) {
    const int r = e / nbw, c = e % nbw;
    Us[r][c] = d.w[(size_t)(k0 + r) * d.ldw + k0 + c];
  }
  __syncthreads();
  if (threadIdx.x < nbw) dinv[threadIdx.x] = zinv(Us[threadIdx.x][threadIdx.x]);
  __syncthreads();
  const int q = blockIdx.x * RB_THREADS + threadIdx.x;
  const int nrhs = d.ncols - s;
  if (q >= nrhs) return;
  const int c = s + q;
  z64* __restrict__ w = d.w;
  const size_t ld = d.ldw;
  z64 x[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nbw) x[j] = w[(size_t)(k0 + j) * ld + c];
#pragma unroll
  for (int j = NB - 1; j >= 0; --j) {
    if (j < nbw) {
      z64 e0 = x[j], e1 = zmk(0.0, 0.0);
#pragma unroll
      for (int i = j + 1; i < NB; ++i)
        if (i < nbw) {
          const z64 u = Us[j][i];
          z64& acc = (i & 1) ? e1 : e0;
          acc.x = fma(-u.x, x[i].x, acc.x);
          acc.x = fma(u.y, x[i].y, acc.x);
          acc.y = fma(-u.x, x[i].y, acc.y);
          acc.y = fma(-u.y, x[i].x, acc.y);
        }
      x[j] = zmul(zadd(e0, e1), dinv[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nbw) w[(size_t)(k0 + j) * ld + c] = x[j];
}
// Hermitian LDL^H panel without pivoting (the factorisation of the sweep
// blocks D_i, which are Hermitian at real E; the paper factors them with a
// no-pivoting Hermitian solver, Sec. 5E).  Only the lower triangle of the
// trailing matrix is kept up to date.  Two launches per panel:
//   herm_diag  one CTA per problem reads the lower triangle of the nb x nb
//              diagonal block, factors it as L11 D1 L11^H in shared memory and
//              writes L11 (strictly lower), D1 (diagonal) and U11 = D1 L11^H
//              (upper) back;
//   herm_rows  CTA x solves its HP_THREADS rows of A21 against U11,
//              L21 = A21 U11^-1, and writes U12 = D1 L21^H (the transposed rows)
//              into the upper triangle.
// The result has the layout of the LU code (unit L below the diagonal, U on
// and above it, no row exchanges), so its right-hand-side solve, trailing
// update (restricted to the lower triangle) and back substitution apply
// unchanged.  A zero or non-finite d_j records 1 + its column in *info.
constexpr int HP_THREADS = 128;
// Largest |re| + |im| of an entry of L accepted from the unpivoted Hermitian
// factorisation; beyond it the pivot growth has used up most of FP64.
constexpr double HERM_MAX_L = 1e8;

template <int NB>
__global__ void __launch_bounds__(HP_THREADS) herm_diag_kernel(const LuDesc* __restrict__ descs, int k0, int nb) {
  const LuDesc d = descs[blockIdx.x];
  if (d.active && __ldg(d.active) == 0) return;
  const int s = d.s;
  if (k0 >= s) return;
  const int nbw = min(min(nb, NB), s - k0);
  z64* __restrict__ w = d.w;
  const size_t ld = d.ldw;
  __shared__ z64 Dg[NB][NB + 1];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < nbw * nbw; e += HP_THREADS) {
    const int i = e / nbw, j = e % nbw;
    if (j <= i) Dg[i][j] = w[(size_t)(k0 + i) * ld + k0 + j];
  }
  __syncthreads();
  for (int j = 0; j < nbw; ++j) {
    const z64 dj = Dg[j][j];
    const z64 inv = zinv(dj);  // zero for a zero pivot (recorded below)
    const int m = nbw - 1 - j;
    // Dg[i][c] -= Dg[i][j] conj(Dg[c][j]) / d_j for j < c <= i (column j still unscaled)
    for (int e = tid; e < m * m; e += HP_THREADS) {
      const int i = j + 1 + e / m, c = j + 1 + e % m;
      if (c <= i) Dg[i][c] = zsub(Dg[i][c], zmul(zmul(Dg[i][j], inv), zconj(Dg[c][j])));
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < nbw; i += HP_THREADS) Dg[i][j] = zmul(Dg[i][j], inv);
    if (tid == 0) {
      const double a = fabs(dj.x) + fabs(dj.y);
      if (bad == 0 && !(a > 0.0 && a <= 1.7976931348623157e308)) bad = j + 1;
    }
    __syncthreads();
  }
  for (int e = tid; e < nbw * nbw; e += HP_THREADS) {
    const int i = e / nbw, j = e % nbw;
    w[(size_t)(k0 + i) * ld + k0 + j] = j <= i ? Dg[i][j] : zmul(Dg[i][i], zconj(Dg[j][i]));
  }
  for (int t = tid; t < nbw; t += HP_THREADS) d.ipiv[k0 + t] = k0 + t;
  if (tid == 0 && bad && d.info && *d.info == 0) *d.info = k0 + bad;
}

template <int NB>
__global__ void __launch_bounds__(HP_THREADS) herm_rows_kernel(const LuDesc* __restrict__ descs, int k0, int nb) {
  const LuDesc d = descs[blockIdx.y];
  if (d.active && __ldg(d.active) == 0) return;
  const int s = d.s;
  if (k0 >= s) return;
  const int nbw = min(min(nb, NB), s - k0);
  const int r = k0 + nbw + blockIdx.x * HP_THREADS + threadIdx.x;
  if (k0 + nbw + blockIdx.x * HP_THREADS >= s) return;  // no rows for this CTA (uniform)
  z64* __restrict__ w = d.w;
  const size_t ld = d.ldw;
  __shared__ z64 Uu[NB][NB + 1];  // U11 = D1 L11^H, upper triangle with the diagonal
  __shared__ z64 dinv[NB];
  for (int e = threadIdx.x; e < nbw * nbw; e += HP_THREADS) {
    const int c = e / nbw, j = e % nbw;
    if (c <= j) Uu[c][j] = w[(size_t)(k0 + c) * ld + k0 + j];
  }
  __syncthreads();
  if (threadIdx.x < nbw) dinv[threadIdx.x] = zinv(Uu[threadIdx.x][threadIdx.x]);
  __syncthreads();
  if (r >= s) return;
  z64 a[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) a[c] = c < nbw ? w[(size_t)r * ld + k0 + c] : zmk(0.0, 0.0);
  // l U11 = a: l_j = (a_j - sum_{c<j} l_c U_cj) / d_j
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < nbw) {
      z64 acc = a[j];
#pragma unroll
      for (int c = 0; c < j; ++c) {
        const z64 u = Uu[c][j];
        acc.x = fma(-a[c].x, u.x, acc.x);
        acc.x = fma(a[c].y, u.y, acc.x);
        acc.y = fma(-a[c].x, u.y, acc.y);
        acc.y = fma(-a[c].y, u.x, acc.y);
      }
      a[j] = zmul(acc, dinv[j]);
    }
  }
  bool grow = false;
#pragma unroll
  for (int c = 0; c < NB; ++c)
    if (c < nbw) {
      w[(size_t)r * ld + k0 + c] = a[c];
      w[(size_t)(k0 + c) * ld + r] = zmul(Uu[c][c], zconj(a[c]));  // U12 = D1 L21^H
      const double m = fabs(a[c].x) + fabs(a[c].y);
      grow = grow || !(m <= HERM_MAX_L);
    }
  // without pivoting a tiny d_j makes L explode: report it as a singular block
  if (grow && d.info) atomicCAS(d.info, 0, k0 + 1);
}
}  // namespace

void launch_herm_panel(const LuDesc* d, int nprob, int k0, int nb, int smax, cudaStream_t st) {
  if (nprob <= 0 || k0 >= smax) return;
  const int rows = smax - k0 - nb;
  dim3 grid(rows > 0 ? (rows + HP_THREADS - 1) / HP_THREADS : 1, nprob);
  if (nb <= 16) {
    herm_diag_kernel<16><<<nprob, HP_THREADS, 0, st>>>(d, k0, nb);
    if (rows > 0) herm_rows_kernel<16><<<grid, HP_THREADS, 0, st>>>(d, k0, nb);
  } else {
    herm_diag_kernel<MAXNB><<<nprob, HP_THREADS, 0, st>>>(d, k0, nb);
    if (rows > 0) herm_rows_kernel<MAXNB><<<grid, HP_THREADS, 0, st>>>(d, k0, nb);
  }
}

int lu_panel_width(int smax) {
  if (smax <= 512) return 16;
  if (smax <= 1024) return 8;
  return 32;
}

void launch_lu_panel(const LuDesc* d, int nprob, int k0, int nb, int smax, cudaStream_t st, int tournament) {
  if (nprob <= 0) return;
  const int h = smax - k0;  // rows of the tallest panel in the group
  constexpr int CL = 8;
  if (tournament) {
    if (nb == 16 && h <= CL * 64) { lu_panel_tslu_kernel<16, CL, 64><<<nprob * CL, 64, 0, st>>>(d, k0, nb); return; }
    if (nb == 16 && h <= CL * 128) { lu_panel_tslu_kernel<16, CL, 128><<<nprob * CL, 128, 0, st>>>(d, k0, nb); return; }
    if (nb == 8 && h <= CL * 64) { lu_panel_tslu_kernel<8, CL, 64><<<nprob * CL, 64, 0, st>>>(d, k0, nb); return; }
    if (nb == 8 && h <= CL * 128) { lu_panel_tslu_kernel<8, CL, 128><<<nprob * CL, 128, 0, st>>>(d, k0, nb); return; }
  }
  if (nb == 16 && h <= CL * 64) lu_panel_cluster_kernel<16, CL, 64><<<nprob * CL, 64, 0, st>>>(d, k0, nb);
  else if (nb == 16 && h <= CL * 128) lu_panel_cluster_kernel<16, CL, 128><<<nprob * CL, 128, 0, st>>>(d, k0, nb);
  else if (nb == 8 && h <= CL * 64) lu_panel_cluster_kernel<8, CL, 64><<<nprob * CL, 64, 0, st>>>(d, k0, nb);
  else if (nb == 8 && h <= CL * 128) lu_panel_cluster_kernel<8, CL, 128><<<nprob * CL, 128, 0, st>>>(d, k0, nb);
  else if (nb <= 16 && h <= PANEL_THREADS) lu_panel_reg_kernel<16, 1><<<nprob, PANEL_THREADS, 0, st>>>(d, k0, nb);
  else if (nb <= 8 && h <= 2 * PANEL_THREADS) lu_panel_reg_kernel<8, 2><<<nprob, PANEL_THREADS, 0, st>>>(d, k0, nb);
  else lu_panel_kernel<<<nprob, PANEL_THREADS, 0, st>>>(d, k0, nb);
}

void launch_lu_rowblock(const LuDesc* d, int nprob, int k0, int nb, int nbo, int far, int max_cols,
                        cudaStream_t st, int max_rows) {
  if (nprob <= 0 || max_cols <= 0) return;
  if (far == 3 && nbo > 0 && max_rows > 0 && exchange_smem(max_rows, nbo) <= XSMEM_MAX) {
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(lu_block_exchange_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XSMEM_MAX);
      attr_set = true;
    }
    dim3 xgrid((max_cols + XC - 1) / XC, nprob);
    lu_block_exchange_kernel<<<xgrid, XT, exchange_smem(max_rows, nbo), st>>>(d, (k0 / nbo) * nbo, nbo);
    return;
  }
  dim3 grid((max_cols + RB_THREADS - 1) / RB_THREADS, nprob);
  if (nb <= 8) lu_rowblock_kernel<8><<<grid, RB_THREADS, 0, st>>>(d, k0, nb, nbo, far);
  else if (nb <= 16) lu_rowblock_kernel<16><<<grid, RB_THREADS, 0, st>>>(d, k0, nb, nbo, far);
  else lu_rowblock_kernel<MAXNB><<<grid, RB_THREADS, 0, st>>>(d, k0, nb, nbo, far);
}

void launch_lu_backsub_diag(const LuDesc* d, int nprob, int k0, int nb, int max_rhs, cudaStream_t st) {
  if (nprob <= 0 || max_rhs <= 0) return;
  dim3 grid((max_rhs + RB_THREADS - 1) / RB_THREADS, nprob);
  if (nb <= 8) lu_backsub_diag_kernel<8><<<grid, RB_THREADS, 0, st>>>(d, k0, nb);
  else if (nb <= 16) lu_backsub_diag_kernel<16><<<grid, RB_THREADS, 0, st>>>(d, k0, nb);
  else lu_backsub_diag_kernel<MAXNB><<<grid, RB_THREADS, 0, st>>>(d, k0, nb);
}

}  // namespace ss
