// C ABI and pipeline of the SplitSolve hot path (see include/splitsolve.h).
//
// Per batch ("chunk") of (E,k) points the pipeline is
//   1. self-energies: Sancho-Rubio doubling on both leads of every point
//      (2 problems per point), iterations replayed from a captured graph until
//      every problem has converged or hit the cap (decimation, Sec. 3A);
//   2. block sweeps: Algorithm 1 for the first block column and its mirror for
//      the last one, both directions of every point in the same launches
//      (Sec. 3B, "two accelerators" become two problem groups on one GPU);
//   3. boundary correction of Eq. x: R = 1 - C Q, LU(R), z, x = Q (b' + z) and
//      the corner G_1n of (A - B C)^-1;
//   4. T = Re Tr[Gamma_L G_1n Gamma_R G_1n^H];
//   5. mixed path with x requested: refinement of x to a normwise backward
//      error <= ir_tol (residual, block-UL correction with the kept D_i^-1,
//      SMW correction with the kept R^-1).
// In the mixed path every product is the exact digit-sliced tensor-core GEMM
// (ss_oz.cu); pivoted panels and triangular blocks of the LU stay FP64.
// Points are ordered longest-first by n_b * s_b^3 and cut into chunks that
// fit the workspace allocated at ss_create (the batch scheduler).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "splitsolve.h"
#include "ss_internal.cuh"
#include "ss_plan.h"
#include "ss_tc.h"

using namespace ss;

namespace {

constexpr int LU_NB = 0;  // panel width chosen per group from its largest block
// Outer block width of the two-level LU in the mixed path: the exact
// tensor-core trailing updates then have depth 128 instead of the panel width.
inline int lu_outer_default(int smax) { return smax >= 256 ? 128 : (smax >= 128 ? 64 : 0); }
constexpr int MAX_K_ID = 4096;
// Learned warm start inside the pipeline: fixed-point steps after the network's
// seed and the Dyson-residual acceptance threshold (cap 8 steps, accept at
// ||g (D - U g L) - 1||_F / sqrt(s) <= 1e-10; doubling otherwise).
constexpr int WARM_ITERS = 8;
constexpr double WARM_TOL = 1e-10;

std::string g_create_error;

struct KData {
  int n = 0, s = 0;
  double kval = 0.0;  // transverse momentum fed to the warm-start network
  z64 *Hd = nullptr, *Hu = nullptr, *Sd = nullptr, *Su = nullptr, *lead = nullptr;
  // lead cells: [side][0..3] = H00, H01, S00, S01
  const z64* cell[2][4] = {{nullptr, nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr, nullptr}};
  void free_all() {
    cudaFree(Hd); cudaFree(Hu); cudaFree(Sd); cudaFree(Su); cudaFree(lead);
    Hd = Hu = Sd = Su = lead = nullptr;
  }
};

struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(char* b) : base(b) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Most partitions a device is split into (Sec. 3B, Fig. pp).
constexpr int MAXP = 8;
// Blocks per point whose diagonal Green's function blocks one round of the
// density-of-states step inverts.
constexpr int DOS_ROUND = 8;

// What the sweeps of a call must keep.
enum Layout {
  LAYOUT_FULL = 0,  // both block columns of every partition (wave functions x)
  LAYOUT_LEAN = 1,  // transmission only: running corner products, no block columns
  LAYOUT_DOS = 2    // density of states: the two sweeps' Schur products of every block
};

// Workspace of one point inside a chunk.
struct PW {
  int idx = 0;  // position in the call's arrays
  int n = 0, s = 0;
  double E = 0.0;
  const KData* kd = nullptr;
  // partitions: np contiguous block ranges [pa[j], pb[j]] (1-based), whose
  // sweeps run concurrently and are merged by one SMW system of 2 np s rows
  int np = 1;
  int pa[MAXP] = {0}, pb[MAXP] = {0};
  Layout layout = LAYOUT_FULL;
  // self-energy doubling, side 0 = left lead, 1 = right lead
  z64 *D[2], *e[2], *es[2], *a[2][2], *b[2][2], *T1[2], *T2[2], *Wd[2];
  int* ipd[2];
  z64* sig[2];
  // sweeps, dir 0 = first block column, 1 = last block column of each partition
  z64* X[2] = {nullptr, nullptr};  // full: the block columns (global block index); dos: Schur products
  z64* Ws[MAXP][2];                // [D_i | RHS (| 1)] work of each sweep
  int* ips[MAXP][2];
  z64* tmp[MAXP][2];               // full: chain product
  z64* Xl[MAXP][2][2];             // lean, dos: ping-pong X_i of the sweep
  z64* Rl[MAXP][2][2];             // lean: ping-pong running corner product
  const z64* Gc[MAXP][4];          // corners of each partition's inverse: G_aa, G_ba, G_ab, G_bb
  // boundary
  z64 *Rw, *gb, *cv, *G1n, *Gam[2], *M1, *M2;
  int* ipr;
  z64* inj = nullptr;  // device copy or user pointer (2s x ninj)
  z64* x = nullptr;    // device output (N x ninj)
  // FP64 iterative refinement of x (mixed mode): D_i^-1 of the first-column
  // sweep, R^-1, residual r, UL-substitution work w, SMW work zc, t
  z64 *Dinv = nullptr, *r = nullptr, *wv = nullptr, *zc = nullptr, *tv = nullptr;
  // density of states: [K_i | 1] of one round of blocks, pivots
  z64* Kw = nullptr;
  int* ipk = nullptr;
  int rows() const { return 2 * np * s; }  // rows of the boundary system
};

// Split n blocks into np contiguous partitions of (almost) equal length.
void set_partitions(PW& w, int parts) {
  w.np = std::max(1, std::min({parts, w.n, MAXP}));
  for (int j = 0; j < w.np; ++j) {
    w.pa[j] = 1 + (int)((long long)j * w.n / w.np);
    w.pb[j] = (int)((long long)(j + 1) * w.n / w.np);
  }
}

// Workspace of one point, in two parts.  The doubling buffers and the
// self-energies of every point of a batch are carved first (carve_doubling),
// so their addresses depend only on the batch's block sizes and cached
// self-energies stay valid whatever the next call's layout, partitions or
// n_inj; the sweep and boundary buffers follow (carve_sweeps).
void carve_doubling(Carve& c, PW& w) {
  const int s = w.s;
  const size_t ss2 = (size_t)s * s;
  for (int q = 0; q < 2; ++q) {
    w.D[q] = c.take<z64>(ss2); w.e[q] = c.take<z64>(ss2); w.es[q] = c.take<z64>(ss2);
    w.a[q][0] = c.take<z64>(ss2); w.a[q][1] = c.take<z64>(ss2);
    w.b[q][0] = c.take<z64>(ss2); w.b[q][1] = c.take<z64>(ss2);
    w.T1[q] = c.take<z64>(ss2); w.T2[q] = c.take<z64>(ss2); w.Wd[q] = c.take<z64>(3 * ss2);
    w.ipd[q] = c.take<int>(s);
    w.sig[q] = c.take<z64>(ss2);
  }
}

void carve_sweeps(Carve& c, PW& w, int ninj, bool ir) {
  const int n = w.n, s = w.s;
  const size_t ss2 = (size_t)s * s;
  const Layout L = w.layout;
  if (L != LAYOUT_LEAN) { w.X[0] = c.take<z64>((size_t)n * ss2); w.X[1] = c.take<z64>((size_t)n * ss2); }
  for (int j = 0; j < w.np; ++j)
    for (int d = 0; d < 2; ++d) {
      w.Ws[j][d] = c.take<z64>(3 * ss2);
      w.ips[j][d] = c.take<int>(s);
      if (L == LAYOUT_FULL) w.tmp[j][d] = c.take<z64>(ss2);
      if (L != LAYOUT_FULL) { w.Xl[j][d][0] = c.take<z64>(ss2); w.Xl[j][d][1] = c.take<z64>(ss2); }
      if (L == LAYOUT_LEAN) { w.Rl[j][d][0] = c.take<z64>(ss2); w.Rl[j][d][1] = c.take<z64>(ss2); }
    }
  if (L == LAYOUT_DOS) {
    const int rb = std::min(n, DOS_ROUND);
    w.Kw = c.take<z64>((size_t)rb * 2 * ss2);
    w.ipk = c.take<int>((size_t)rb * s);
    return;
  }
  const int S2 = w.rows();
  const int nj = L == LAYOUT_FULL ? ninj : 0;
  const bool irr = ir && L == LAYOUT_FULL;
  const int ldr = S2 + s + nj + (irr ? S2 : 0);
  w.Rw = c.take<z64>((size_t)S2 * ldr);
  w.G1n = c.take<z64>(ss2);
  w.Gam[0] = c.take<z64>(ss2); w.Gam[1] = c.take<z64>(ss2); w.M1 = c.take<z64>(ss2); w.M2 = c.take<z64>(ss2);
  w.ipr = c.take<int>(S2);
  if (L == LAYOUT_FULL) {
    w.gb = c.take<z64>((size_t)S2 * ninj);
    w.cv = c.take<z64>((size_t)S2 * ninj);
    w.inj = c.take<z64>((size_t)2 * s * ninj);
    w.x = c.take<z64>((size_t)n * s * ninj);
  }
  if (irr) {
    w.Dinv = c.take<z64>((size_t)n * ss2);
    w.r = c.take<z64>((size_t)n * s * ninj);
    w.wv = c.take<z64>((size_t)n * s * ninj);
    w.zc = c.take<z64>((size_t)S2 * ninj);
    w.tv = c.take<z64>((size_t)S2 * ninj);
  }
}

// Carve a batch: every point's doubling part, then every point's sweep part.
void carve_batch(Carve& c, std::vector<PW>& pts, int ninj, bool ir) {
  for (auto& w : pts) carve_doubling(c, w);
  for (auto& w : pts) carve_sweeps(c, w, ninj, ir);
}

size_t point_bytes(int n, int s, int ninj, bool ir, Layout layout, int parts) {
  Carve c(nullptr);
  std::vector<PW> one(1);
  one[0].n = n; one[0].s = s; one[0].layout = layout;
  set_partitions(one[0], parts);
  carve_batch(c, one, ninj, ir);
  return c.off + 512;
}

// ------------------------------------------------------------ descriptors
Operand plain(const z64* p, int ld, int trans = 0) {
  Operand o{};
  o.p = p; o.s = nullptr; o.e = make_double2(0.0, 0.0); o.ld = ld; o.trans = trans;
  return o;
}
Operand formed(const z64* S, const z64* H, z64 e, int ld, int trans = 0) {
  Operand o{};
  o.p = H; o.s = S; o.e = e; o.ld = ld; o.trans = trans;
  return o;
}
GemmDesc gdesc(int m, int n, int k, Operand a, Operand b, z64* c, int ldc, z64 alpha, z64 beta,
               const int* active = nullptr) {
  GemmDesc g{};
  g.m = m; g.n = n; g.k = k; g.a = a; g.b = b; g.c = c; g.ldc = ldc; g.cmode = 0;
  g.alpha = alpha; g.beta = beta; g.active = active;
  return g;
}
FormDesc fdesc(z64* out, int ldo, int rows, int cols) {
  FormDesc f{};
  f.out = out; f.ldo = ldo; f.rows = rows; f.cols = cols;
  f.ax = f.ay = f.az = f.gamma = make_double2(0.0, 0.0);
  return f;
}
FormDesc fcopy(z64* out, int ldo, const z64* in, int ldi, int rows, int cols, int trans = 0) {
  FormDesc f = fdesc(out, ldo, rows, cols);
  f.x = in; f.ldx = ldi; f.tx = trans; f.ax = make_double2(1.0, 0.0);
  return f;
}
// out = e * op(S) - op(H)
FormDesc fformed(z64* out, int ldo, const z64* S, const z64* H, z64 e, int ld, int rows, int cols,
                 int trans = 0) {
  FormDesc f = fdesc(out, ldo, rows, cols);
  f.x = S; f.ldx = ld; f.tx = trans; f.ax = e;
  f.y = H; f.ldy = ld; f.ty = trans; f.ay = make_double2(-1.0, 0.0);
  return f;
}
FormDesc fident(z64* out, int ldo, int rows, int cols, double g) {
  FormDesc f = fdesc(out, ldo, rows, cols);
  f.gamma = make_double2(g, 0.0);
  return f;
}

const z64 ONE = {1.0, 0.0}, ZERO = {0.0, 0.0}, MONE = {-1.0, 0.0};

}  // namespace

// --------------------------------------------------------------- the handle
struct ss_handle {
  ss_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  std::map<int, KData> ks;
  std::string err;
  long long nlaunch = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  // per-chunk device scalars
  int* dint = nullptr;      // flags, iterations, infos
  double* ddbl = nullptr;   // norms
  z64* dtr = nullptr;       // traces
  size_t dint_n = 0, ddbl_n = 0, dtr_n = 0;
  Plan p_setup, p_iter[2], p_final, p_sweep, p_bound;
  Prof prof;
  // mixed path: packing buffer of the tensor-core GEMMs and their error flag
  unsigned char* pack = nullptr;
  size_t pack_bytes = 0;
  int* tc_err = nullptr;
  bool mixed() const { return cfg.precision != SS_FP64; }
  bool plan_error = false;  // a tensor-core group did not fit the packing buffer
  // learned warm start
  ss_mlp* warm_net[2] = {nullptr, nullptr};
  double warm_scale[2] = {1.0, 1.0};
  float* feat = nullptr;    // max_points x n_in features
  float* warm_y = nullptr;  // max_points x n_out network outputs
  double* wres = nullptr;   // per-point Dyson residual (sum of squares)
  size_t warm_cap = 0;
  Plan p_warm_iter, p_warm_judge, p_final_g;
  Plan p_ir_res, p_ir_cor;
  // autotuned LU settings per block size: panel width and update arithmetic
  struct Tune { int nb; int nbo; int upd; double ms; int gsq = -1; int gup = -1; };
  std::map<int, Tune> tune;
  std::vector<double> c_err;  // normwise backward error of the last refined solve
  Prof* P() { return cfg.profile ? &prof : nullptr; }
  // cache of the last chunk
  std::vector<double> cE;
  std::vector<int> cK;
  bool c_sigma = false, c_T = false;
  std::vector<double> cT, cTi;
  std::vector<int> c_iters, c_status;
  long long nhost = 0;  // host-side launch calls (eager kernels, memsets, graph launches)
  // contour-integral (FEAST) open boundary conditions: scratch and plans
  char* feast_buf = nullptr;
  size_t feast_bytes = 0;
  int* feast_info = nullptr;
  size_t feast_info_n = 0;
  Plan p_fa, p_fb, p_fc;
};

namespace {

int fail(ss_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}
int cuda_fail(ss_handle* h, cudaError_t e, const char* where) {
  return fail(h, SS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(call, where)                              \
  do {                                               \
    cudaError_t _e = (call);                         \
    if (_e != cudaSuccess) return cuda_fail(h, _e, where); \
  } while (0)

// A group of large GEMMs: the FP64 kernel, or in the mixed mode the
// FP64-accurate digit-sliced kernel on the tensor cores.
bool big_gemm(ss_handle* h, Plan& P, const std::vector<GemmDesc>& g) {
  if (g.empty()) return true;
  if (!h->mixed()) { P.gemm(g); return true; }
  if (!P.oz_gemm(g, h->pack, h->pack_bytes, h->tc_err)) {
    h->plan_error = true;
    return false;
  }
  return true;
}
void lu(ss_handle* h, Plan& P, const std::vector<LuDesc>& ds) {
  int smax = 0;
  for (auto& d : ds) smax = std::max(smax, d.s);
  int nb = LU_NB, nbo = h->mixed() ? lu_outer_default(smax) : 0;
  Plan::Updates upd = h->mixed() ? Plan::UPD_EXACT_TC : Plan::UPD_FP64;
  auto it = h->tune.find(smax);
  if (it != h->tune.end()) { nb = it->second.nb; nbo = it->second.nbo; upd = (Plan::Updates)it->second.upd; }
  if (!P.lu_solve(ds, nb, upd, h->pack, h->pack_bytes, h->tc_err, nbo, h->cfg.tournament_pivoting,
                  h->cfg.lu_lookahead))
    h->plan_error = true;
}
// The sweep blocks D_i with cfg.hermitian_sweeps: LDL^H without pivoting,
// updates on the lower triangle (FP64 path: FP64 updates of depth 16; mixed
// path: exact tensor-core updates of depth 32).
void ldl(ss_handle* h, Plan& P, const std::vector<LuDesc>& ds) {
  const bool mx = h->mixed();
  if (!P.ldl_solve(ds, mx ? 32 : 16, mx ? Plan::UPD_EXACT_TC : Plan::UPD_FP64, h->pack, h->pack_bytes, h->tc_err))
    h->plan_error = true;
}

// ---------------------------------------------------------- self-energies
// Builds setup / iteration / final plans for the doubling of 2P lead problems.
// seeded (optional, 2 per point): 1 where an accepted warm start already holds
// the lead's surface Green's function g in es[q]; that lead skips the doubling
// (its flag starts at 0) and its self-energy is A_{1,0} g A_{0,1} (left) or
// A_{n,n+1} g A_{n+1,n} (right).
void build_decimation(ss_handle* h, std::vector<PW>& pts, int* act, int* iters, int* conv,
                      int* info, double* na, double* nb, double* nd, bool preset_act = false,
                      const std::vector<int>* seeded = nullptr) {
  const int P = (int)pts.size();
  const int NP = 2 * P;
  const double eta = h->cfg.eta;
  auto is_seeded = [&](int i) { return seeded && (*seeded)[i] != 0; };
  Plan& S = h->p_setup;
  S.clear();
  std::vector<FormDesc> f;
  std::vector<Norm1Desc> nD, nA;
  for (int p = 0; p < P; ++p) {
    PW& w = pts[p];
    const int s = w.s;
    const z64 z = make_double2(w.E, eta);
    for (int q = 0; q < 2; ++q) {
      if (is_seeded(2 * p + q)) continue;
      const z64* const* c = w.kd->cell[q];
      f.push_back(fformed(w.D[q], s, c[2], c[0], z, s, s, s));
      f.push_back(fformed(w.e[q], s, c[2], c[0], z, s, s, s));
      f.push_back(fformed(w.es[q], s, c[2], c[0], z, s, s, s));
      f.push_back(fformed(w.a[q][0], s, c[3], c[1], z, s, s, s));
      // L = z S01^H - H01^H
      f.push_back(fformed(w.b[q][0], s, c[3], c[1], z, s, s, s, 1));
    }
  }
  S.form(f);
  S.memset0(na, sizeof(double) * NP);
  S.memset0(nb, sizeof(double) * NP);
  S.memset0(nd, sizeof(double) * NP);
  if (!preset_act) S.fill(act, NP, 1);
  S.memset0(iters, sizeof(int) * NP);
  S.memset0(conv, sizeof(int) * NP);
  S.memset0(info, sizeof(int) * NP * 2);
  for (int p = 0; p < P; ++p) {
    PW& w = pts[p];
    for (int q = 0; q < 2; ++q) {
      const int i = 2 * p + q;
      if (is_seeded(i)) continue;
      nD.push_back({w.D[q], w.s, w.s, w.s, nd + i, nullptr});
      nA.push_back({w.a[q][0], w.s, w.s, w.s, na + i, nullptr});
      nA.push_back({w.b[q][0], w.s, w.s, w.s, nb + i, nullptr});
    }
  }
  S.norm1(nD);
  S.norm1(nA);
  S.check(na, nb, nd, act, iters, conv, NP, h->cfg.decim_tol, h->cfg.decim_max_iter, 0);

  for (int ping = 0; ping < 2; ++ping) {
    Plan& I = h->p_iter[ping];
    I.clear();
    const int pong = 1 - ping;
    std::vector<FormDesc> f1, f2;
    std::vector<LuDesc> lu;
    std::vector<GemmDesc> g;
    std::vector<Norm1Desc> nr;
    for (int p = 0; p < P; ++p) {
      PW& w = pts[p];
      const int s = w.s, ld = 3 * s;
      for (int q = 0; q < 2; ++q) {
        const int i = 2 * p + q;
        const int* ac = act + i;
        z64* W = w.Wd[q];
        FormDesc x;
        x = fcopy(W, ld, w.e[q], s, s, s); x.active = ac; f1.push_back(x);
        x = fcopy(W + s, ld, w.a[q][ping], s, s, s); x.active = ac; f1.push_back(x);
        x = fcopy(W + 2 * s, ld, w.b[q][ping], s, s, s); x.active = ac; f1.push_back(x);
        LuDesc L{};
        L.w = W; L.ldw = ld; L.s = s; L.ncols = 3 * s; L.ipiv = w.ipd[q]; L.info = info + i;
        L.active = ac;
        lu.push_back(L);
        const z64* ga = W + s;
        const z64* gbp = W + 2 * s;
        g.push_back(gdesc(s, s, s, plain(w.a[q][ping], s), plain(gbp, ld), w.T1[q], s, ONE, ZERO, ac));
        g.push_back(gdesc(s, s, s, plain(w.b[q][ping], s), plain(ga, ld), w.T2[q], s, ONE, ZERO, ac));
        g.push_back(gdesc(s, s, s, plain(w.a[q][ping], s), plain(ga, ld), w.a[q][pong], s, MONE, ZERO, ac));
        g.push_back(gdesc(s, s, s, plain(w.b[q][ping], s), plain(gbp, ld), w.b[q][pong], s, MONE, ZERO, ac));
        // e -= T1 + T2 ; es_R -= T1 (right lead) or es_L -= T2 (left lead)
        FormDesc u = fcopy(w.e[q], s, w.e[q], s, s, s);
        u.y = w.T1[q]; u.ldy = s; u.ay = MONE;
        u.z = w.T2[q]; u.ldz = s; u.az = MONE;
        u.active = ac;
        f2.push_back(u);
        FormDesc v = fcopy(w.es[q], s, w.es[q], s, s, s);
        v.y = (q == 1) ? w.T1[q] : w.T2[q]; v.ldy = s; v.ay = MONE;
        v.active = ac;
        f2.push_back(v);
        nr.push_back({w.a[q][pong], s, s, s, na + i, ac});
        nr.push_back({w.b[q][pong], s, s, s, nb + i, ac});
      }
    }
    I.form(f1);
    ::lu(h, I, lu);
    big_gemm(h, I, g);
    I.form(f2);
    I.norm1(nr);
    I.check(na, nb, nd, act, iters, conv, NP, h->cfg.decim_tol, h->cfg.decim_max_iter, 1);
  }

  // Sigma_L = A_{1,0} es_L^-1 A_{0,1};  Sigma_R = A_{n,n+1} es_R^-1 A_{n+1,n}
  Plan& F = h->p_final;
  F.clear();
  std::vector<FormDesc> ff;
  std::vector<LuDesc> lu;
  std::vector<GemmDesc> g;
  std::vector<GemmDesc> gs;
  for (int p = 0; p < P; ++p) {
    PW& w = pts[p];
    const int s = w.s, ld = 3 * s;
    const z64 E = make_double2(w.E, 0.0);
    for (int q = 0; q < 2; ++q) {
      const z64* const* c = w.kd->cell[q];
      z64* W = w.Wd[q];
      if (is_seeded(2 * p + q)) {
        // W + s = g A (seeded g), in place of the solve es W = A below
        gs.push_back(gdesc(s, s, s, plain(w.es[q], s), formed(c[3], c[1], E, s, q == 1 ? 1 : 0), W + s, ld, ONE, ZERO));
      } else {
        ff.push_back(fcopy(W, ld, w.es[q], s, s, s));
        // right: rhs A_{n+1,n} = (E S01 - H01)^H ; left: rhs A_{0,1} = E S01 - H01
        ff.push_back(fformed(W + s, ld, c[3], c[1], E, s, s, s, q == 1 ? 1 : 0));
        LuDesc L{};
        L.w = W; L.ldw = ld; L.s = s; L.ncols = 2 * s; L.ipiv = w.ipd[q]; L.info = info + NP + 2 * p + q;
        lu.push_back(L);
      }
      g.push_back(gdesc(s, s, s, formed(c[3], c[1], E, s, q == 1 ? 0 : 1), plain(W + s, ld), w.sig[q], s,
                        ONE, ZERO));
    }
  }
  F.form(ff);
  ::lu(h, F, lu);
  big_gemm(h, F, gs);
  big_gemm(h, F, g);
}

// Warm start of lead `side` for the points of one batch (all of block size
// s = sqrt(n_out / 2) of the attached network): network seed g0 = MLP(E, k),
// at most `iters` steps of g <- (D - U g L)^-1 (right lead; (D - L g U)^-1
// left), then the FP64 Dyson residual ||g (D - U g L) - 1||_F / sqrt(s); a
// point is accepted when it is <= tol, with g left in es[side].
// Returns SS_OK or a call-level error; accepted[p] on the host.
int warm_seed(ss_handle* h, std::vector<PW>& pts, int side, const std::vector<double>& kvals, int iters,
              double tol, int* dinfo, std::vector<int>& accepted) {
  ss_mlp* net = h->warm_net[side];
  const int P = (int)pts.size();
  accepted.assign(P, 0);
  if (!net || P == 0) return SS_OK;
  int n_in = 0, n_out = 0, mb = 0;
  mlp_dims(net, &n_in, &n_out, &mb);
  const int s = pts[0].s;
  for (auto& w : pts)
    if (w.s != s || 2 * s * s != n_out) return fail(h, SS_ERR_ARG, "network output does not match s_b");
  if (P > mb) return fail(h, SS_ERR_ARG, "network max_batch below max_points");
  cudaStream_t st = h->stream;
  const double eta = h->cfg.eta;
  const int P_max = h->cfg.max_points;
  const size_t need = (size_t)P_max * (n_in + n_out);
  if (need > h->warm_cap) {
    cudaFree(h->feat); cudaFree(h->warm_y); cudaFree(h->wres);
    h->feat = nullptr; h->warm_y = nullptr; h->wres = nullptr;
    CK(cudaMalloc(&h->feat, (size_t)P_max * n_in * sizeof(float)), "warm features");
    CK(cudaMalloc(&h->warm_y, (size_t)P_max * n_out * sizeof(float)), "warm outputs");
    CK(cudaMalloc(&h->wres, (size_t)P_max * sizeof(double)), "warm residuals");
    h->warm_cap = need;
  }
  std::vector<float> f((size_t)P * n_in, 0.f);
  for (int p = 0; p < P; ++p) {
    const double e = pts[p].E, k = kvals[p];
    float* r = &f[(size_t)p * n_in];
    r[0] = (float)e; r[1] = (float)std::cos(k); r[2] = (float)std::sin(k);
    for (int m = 1; m <= 8 && 3 + 2 * m - 1 < n_in; ++m) {
      r[3 + 2 * (m - 1)] = (float)std::sin(m * M_PI * e);
      r[4 + 2 * (m - 1)] = (float)std::cos(m * M_PI * e);
    }
  }
  cudaStream_t ns = mlp_stream(net);
  CK(cudaMemcpyAsync(h->feat, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice, ns), "features");
  int r2 = ss_mlp_forward(net, P, h->feat, h->warm_y);
  if (r2 != SS_OK) return fail(h, r2, "network forward failed");
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
  cudaEventRecord(ev, ns);
  cudaStreamWaitEvent(st, ev, 0);
  cudaEventDestroy(ev);
  for (int p = 0; p < P; ++p) {
    launch_unpack_g(h->warm_y + (size_t)p * n_out, s, 1.0 / h->warm_scale[side], pts[p].es[side], s, st);
    ++h->nlaunch;
  }
  // lead blocks at z and one fixed-point step g <- (D - U g L)^-1 (right) / (D - L g U)^-1 (left)
  Plan& setup = h->p_setup;
  setup.clear();
  std::vector<FormDesc> fl;
  for (auto& w : pts) {
    const z64 z = make_double2(w.E, eta);
    const z64* const* cc = w.kd->cell[side];
    fl.push_back(fformed(w.D[side], s, cc[2], cc[0], z, s, s, s));
    fl.push_back(fformed(w.a[side][0], s, cc[3], cc[1], z, s, s, s));
    fl.push_back(fformed(w.b[side][0], s, cc[3], cc[1], z, s, s, s, 1));
  }
  setup.form(fl);
  Plan& I = h->p_warm_iter;
  I.clear();
  std::vector<GemmDesc> g1, g2;
  std::vector<FormDesc> f1, f2;
  std::vector<LuDesc> lus;
  for (int p = 0; p < P; ++p) {
    PW& w = pts[p];
    const z64* first = side == 1 ? w.a[side][0] : w.b[side][0];
    const z64* second = side == 1 ? w.b[side][0] : w.a[side][0];
    z64* W = w.Wd[side];
    g1.push_back(gdesc(s, s, s, plain(first, s), plain(w.es[side], s), w.T1[side], s, ONE, ZERO));
    f1.push_back(fcopy(W, 2 * s, w.D[side], s, s, s));
    f1.push_back(fident(W + s, 2 * s, s, s, 1.0));
    g2.push_back(gdesc(s, s, s, plain(w.T1[side], s), plain(second, s), W, 2 * s, MONE, ONE));
    LuDesc L{};
    L.w = W; L.ldw = 2 * s; L.s = s; L.ncols = 2 * s; L.ipiv = w.ipd[side]; L.info = dinfo + 2 * p + side;
    lus.push_back(L);
    f2.push_back(fcopy(w.es[side], s, W + s, 2 * s, s, s));
  }
  I.memset0(dinfo, sizeof(int) * 4 * P);
  big_gemm(h, I, g1);
  I.form(f1);
  big_gemm(h, I, g2);
  ::lu(h, I, lus);
  I.form(f2);
  // judge: ||g (D - U g L) - 1||_F^2 into wres, in FP64 whatever the precision mode
  Plan& J = h->p_warm_judge;
  J.clear();
  std::vector<GemmDesc> j1, j2, j3;
  std::vector<FormDesc> jf;
  std::vector<Norm1Desc> fr;
  J.memset0(h->wres, sizeof(double) * P);
  for (int p = 0; p < P; ++p) {
    PW& w = pts[p];
    const z64* first = side == 1 ? w.a[side][0] : w.b[side][0];
    const z64* second = side == 1 ? w.b[side][0] : w.a[side][0];
    z64* W = w.Wd[side];
    j1.push_back(gdesc(s, s, s, plain(first, s), plain(w.es[side], s), w.T1[side], s, ONE, ZERO));
    jf.push_back(fcopy(W, s, w.D[side], s, s, s));
    j2.push_back(gdesc(s, s, s, plain(w.T1[side], s), plain(second, s), W, s, MONE, ONE));
    GemmDesc q = gdesc(s, s, s, plain(w.es[side], s), plain(W, s), w.T2[side], s, ONE, MONE);
    q.cmode = 2;
    j3.push_back(q);
    fr.push_back({w.T2[side], s, s, s, h->wres + p, nullptr});
  }
  J.gemm(j1);
  J.form(jf);
  J.gemm(j2);
  J.gemm(j3);
  J.frob2(fr);
  if (h->plan_error) return fail(h, SS_ERR_OOM, "tensor-core packing buffer too small");
  CK(setup.upload(st), "upload warm");
  CK(I.upload(st), "upload warm");
  CK(J.upload(st), "upload warm");
  CK(setup.run(st, &h->nlaunch, h->P()), "warm setup");
  for (int it = 0; it < iters; ++it) CK(I.run(st, &h->nlaunch, h->P()), "warm step");
  CK(J.run(st, &h->nlaunch, h->P()), "warm judge");
  std::vector<double> res(P);
  std::vector<int> info(2 * P);
  CK(cudaMemcpyAsync(res.data(), h->wres, sizeof(double) * P, cudaMemcpyDeviceToHost, st), "read residual");
  CK(cudaMemcpyAsync(info.data(), dinfo, sizeof(int) * 2 * P, cudaMemcpyDeviceToHost, st), "read info");
  CK(cudaStreamSynchronize(st), "warm sync");
  for (int p = 0; p < P; ++p)
    accepted[p] = (std::isfinite(res[p]) && std::sqrt(res[p] / (double)s) <= tol && info[2 * p + side] == 0) ? 1 : 0;
  return SS_OK;
}

// ------------------------------------------------------------------ sweeps
// Longest partition of the chunk: the number of sequential sweep steps.
int sweep_steps(const std::vector<PW>& pts) {
  int m = 0;
  for (auto& w : pts)
    for (int j = 0; j < w.np; ++j) m = std::max(m, w.pb[j] - w.pa[j] + 1);
  return m;
}
size_t sinfo_index(int p, int j, int dir, int t, int nsteps) {
  return ((size_t)(p * MAXP + j) * 2 + dir) * nsteps + t;
}

// Algorithm 1 (first block column) and its mirror (last block column) of the
// inverse of every partition A_j = A[a..b, a..b] of every point, all in the same
// launches (Sec. 3B: the two columns, and the partitions, are independent).
// Inside a partition the neighbours outside it do not exist: A_{a,a-1} := 1
// for the first column, A_{b,b+1} := 1 for the last.
//   full layout: X_i is stored, then the chains Q_i = -X_i Q_{i-1} overwrite it;
//   lean layout: only the corners are kept.  G_aa = X_a is the sweep's last
//     X, and G_ba = Q_b = (-1)^(L-1) X_b X_{b-1} ... X_a is accumulated while
//     the sweep runs (R <- -R X_i, one product per block as in the chain, but
//     in the next step's launch and with no block column in memory); the
//     mirror gives G_bb and G_ab the same way.
// with_inv: the first-column sweep also returns D_i^-1 (refinement of x).
void build_sweeps(ss_handle* h, std::vector<PW>& pts, int* info, int nsteps, bool with_inv) {
  Plan& S = h->p_sweep;
  S.clear();
  const int P = (int)pts.size();
  S.memset0(info, sizeof(int) * 2 * MAXP * (size_t)P * nsteps);
  for (int t = 0; t <= nsteps; ++t) {  // t = nsteps: the lean layout's last running products
    std::vector<GemmDesc> g;
    std::vector<FormDesc> f, fc;
    std::vector<LuDesc> lu;
    for (int p = 0; p < P; ++p) {
      PW& w = pts[p];
      const int s = w.s;
      const KData* kd = w.kd;
      const size_t ss2 = (size_t)s * s;
      const z64 E = make_double2(w.E, 0.0);
      const bool lean = w.layout == LAYOUT_LEAN;
      for (int j = 0; j < w.np; ++j) {
        const int a = w.pa[j], b = w.pb[j], len = b - a + 1;
        for (int dir = 0; dir < 2; ++dir) {
          if (lean && t >= 2 && t <= len) {
            // running corner product of step t-1: R_{t-1} = -R_{t-2} X_{t-1} (R_0 = X_0)
            const z64* Rp = (t == 2) ? w.Xl[j][dir][0] : w.Rl[j][dir][t & 1];
            g.push_back(gdesc(s, s, s, plain(Rp, s), plain(w.Xl[j][dir][(t - 1) & 1], s), w.Rl[j][dir][(t - 1) & 1],
                              s, MONE, ZERO));
          }
          if (t >= len) continue;
          const int i = dir == 0 ? b - t : a + t;  // 1-based block
          const bool inv = with_inv && dir == 0;
          const int ld = inv ? 3 * s : 2 * s;
          z64* W = w.Ws[j][dir];
          const z64* Sii = kd->Sd + (i - 1) * ss2;
          const z64* Hii = kd->Hd + (i - 1) * ss2;
          if (t == 0) {
            f.push_back(fformed(W, ld, Sii, Hii, E, s, s, s));
          } else {
            // D_i = A_ii - A_{i,i+1} X_{i+1} (first) or A_ii - A_{i,i-1} Y_{i-1} (last)
            const int up = dir == 0 ? i - 1 : i - 2;  // 0-based upper block index
            const z64* Xp = lean ? w.Xl[j][dir][(t - 1) & 1] : w.X[dir] + (size_t)(dir == 0 ? i : i - 2) * ss2;
            GemmDesc q = gdesc(s, s, s, formed(kd->Su + up * ss2, kd->Hu + up * ss2, E, s, dir == 0 ? 0 : 1),
                               plain(Xp, s), W, ld, MONE, ONE);
            q.cmode = 1; q.cs = Sii; q.ch = Hii; q.ce = E; q.ldcf = s;
            g.push_back(q);
          }
          // right-hand side: A_{i,i-1} (first, 1 at i = a) / A_{i,i+1} (last, 1 at i = b)
          if (dir == 0) {
            if (i > a) f.push_back(fformed(W + s, ld, kd->Su + (i - 2) * ss2, kd->Hu + (i - 2) * ss2, E, s, s, s, 1));
            else f.push_back(fident(W + s, ld, s, s, 1.0));
          } else {
            if (i < b) f.push_back(fformed(W + s, ld, kd->Su + (i - 1) * ss2, kd->Hu + (i - 1) * ss2, E, s, s, s, 0));
            else f.push_back(fident(W + s, ld, s, s, 1.0));
          }
          if (inv) f.push_back(fident(W + 2 * s, ld, s, s, 1.0));
          LuDesc L{};
          L.w = W; L.ldw = ld; L.s = s; L.ncols = inv ? 3 * s : 2 * s; L.ipiv = w.ips[j][dir];
          L.info = info + sinfo_index(p, j, dir, t, nsteps);
          lu.push_back(L);
          z64* Xo = lean ? w.Xl[j][dir][t & 1] : w.X[dir] + (size_t)(i - 1) * ss2;
          fc.push_back(fcopy(Xo, s, W + s, ld, s, s));
          if (inv) fc.push_back(fcopy(w.Dinv + (size_t)(i - 1) * ss2, s, W + 2 * s, ld, s, s));
        }
      }
    }
    big_gemm(h, S, g);
    S.form(f);
    // D_i is Hermitian at real E (a Schur complement of the Hermitian A)
    if (h->cfg.hermitian_sweeps) ::ldl(h, S, lu);
    else ::lu(h, S, lu);
    S.form(fc);
  }
  for (auto& w : pts) {
    if (w.layout != LAYOUT_LEAN) continue;
    for (int j = 0; j < w.np; ++j) {
      const int len = w.pb[j] - w.pa[j] + 1;
      const int last = (len - 1) & 1;
      w.Gc[j][0] = w.Xl[j][0][last];                              // G_aa = X_a
      w.Gc[j][1] = len == 1 ? w.Xl[j][0][0] : w.Rl[j][0][last];   // G_ba
      w.Gc[j][2] = len == 1 ? w.Xl[j][1][0] : w.Rl[j][1][last];   // G_ab
      w.Gc[j][3] = w.Xl[j][1][last];                              // G_bb = Y_b
    }
  }
  // full layout: chains Q_i = -X_i Q_{i-1} (first), P_i = -Y_i P_{i+1} (last)
  for (int t = 1; t < nsteps; ++t) {
    std::vector<GemmDesc> g;
    std::vector<FormDesc> fc;
    for (auto& w : pts) {
      if (w.layout != LAYOUT_FULL) continue;
      const int s = w.s;
      const size_t ss2 = (size_t)s * s;
      for (int j = 0; j < w.np; ++j) {
        const int a = w.pa[j], b = w.pb[j];
        if (t > b - a) continue;
        for (int dir = 0; dir < 2; ++dir) {
          const int i = dir == 0 ? a + t : b - t;
          const int prev = dir == 0 ? i - 1 : i + 1;
          g.push_back(gdesc(s, s, s, plain(w.X[dir] + (i - 1) * ss2, s), plain(w.X[dir] + (prev - 1) * ss2, s),
                            w.tmp[j][dir], s, MONE, ZERO));
          fc.push_back(fcopy(w.X[dir] + (i - 1) * ss2, s, w.tmp[j][dir], s, s, s));
        }
      }
    }
    big_gemm(h, S, g);
    S.form(fc);
  }
  for (auto& w : pts) {
    if (w.layout != LAYOUT_FULL) continue;
    const size_t ss2 = (size_t)w.s * w.s;
    for (int j = 0; j < w.np; ++j) {
      w.Gc[j][0] = w.X[0] + (size_t)(w.pa[j] - 1) * ss2;
      w.Gc[j][1] = w.X[0] + (size_t)(w.pb[j] - 1) * ss2;
      w.Gc[j][2] = w.X[1] + (size_t)(w.pa[j] - 1) * ss2;
      w.Gc[j][3] = w.X[1] + (size_t)(w.pb[j] - 1) * ss2;
    }
  }
}

// ---------------------------------------------------------------- boundary
// The merged boundary system of Eq. x.  With np partitions, A - Sigma =
// blockdiag(A_1 .. A_np) + B K' B^T, where B selects the first and last block
// of every partition ("slots" 2j and 2j+1 for partition j) and K' holds
// -Sigma_L (slot 0), -Sigma_R (slot 2 np - 1) and the couplings A_{b_j,b_j+1}
// between neighbouring partitions (slots 2j+1 -> 2j+2 and back); np = 1 is
// SplitSolve's Sigma^RB = B C.  SMW then gives
//   R = 1 + K' g (g = B^T Q: the corners of every partition's inverse),
//   z = -R^-1 K' g b'',  x = Q (b'' + z),  (A - Sigma)^-1 B = Q R^-1,
// so G_1n = (g R^-1)[slot 0, slot 2np-1] and the partitions are merged by one
// 2 np s system (the SPIKE-style merge of Sec. 3B, Fig. pp, in one step).
struct KTerm {
  int t;       // slot partner of the row slot
  Operand op;  // K'(r, t) = alpha op
  z64 alpha;
};
KTerm kterm(const PW& w, int r) {
  const int S = 2 * w.np;
  const size_t ss2 = (size_t)w.s * w.s;
  const z64 E = make_double2(w.E, 0.0);
  if (r == 0) return {0, plain(w.sig[0], w.s), MONE};
  if (r == S - 1) return {S - 1, plain(w.sig[1], w.s), MONE};
  if (r & 1) {  // last block b_j of partition j couples to the first block of j+1
    const int bj = w.pb[r / 2];
    return {r + 1, formed(w.kd->Su + (bj - 1) * ss2, w.kd->Hu + (bj - 1) * ss2, E, w.s), ONE};
  }
  const int bj = w.pb[r / 2 - 1];  // first block a_j couples back to b_{j-1}
  return {r - 1, formed(w.kd->Su + (bj - 1) * ss2, w.kd->Hu + (bj - 1) * ss2, E, w.s, 1), ONE};
}
inline z64 zneg(z64 a) { return make_double2(-a.x, -a.y); }
// Leading dimension of the boundary system [R | E_last | z rhs | (R^-1 rhs)].
inline int bound_ld(const PW& w, int nj, bool irr) { return w.rows() + w.s + nj + (irr ? w.rows() : 0); }

void build_boundary(ss_handle* h, std::vector<PW>& pts, int ninj, int* info, z64* traces, bool ir) {
  Plan& B = h->p_bound;
  B.clear();
  const int P = (int)pts.size();
  B.memset0(info, sizeof(int) * P);
  std::vector<FormDesc> f0, fc, fg;
  std::vector<GemmDesc> gR, gbA, gbB, gsb, gG1, gG2, gx1, gx2, gM;
  std::vector<LuDesc> lu;
  std::vector<TraceDesc> tr;
  for (int p = 0; p < P; ++p) {
    PW& w = pts[p];
    const int s = w.s, S2 = w.rows(), NS = 2 * w.np;
    const int nj = w.layout == LAYOUT_FULL ? ninj : 0;
    const bool irr = ir && nj > 0;
    const int ld = bound_ld(w, nj, irr);
    const size_t ss2 = (size_t)s * s;
    z64* R = w.Rw;
    f0.push_back(fident(R, ld, S2, S2, 1.0));                              // R = 1
    f0.push_back(fident(R + S2, ld, S2 - s, s, 0.0));                      // E_last = [0; ..; 0; 1]
    f0.push_back(fident(R + (size_t)(S2 - s) * ld + S2, ld, s, s, 1.0));   // (disjoint rows: one launch)
    if (nj > 0) f0.push_back(fident(R + S2 + s, ld, S2, nj, 0.0));         // z right-hand side
    if (irr) f0.push_back(fident(R + S2 + s + nj, ld, S2, S2, 1.0));       // R^-1 for the refinement
    // R += K' g: row slot r meets its partner t, whose partition holds two column slots
    for (int r = 0; r < NS; ++r) {
      const KTerm k = kterm(w, r);
      const int jt = k.t / 2, ut = k.t % 2;
      for (int v = 0; v < 2; ++v)
        gR.push_back(gdesc(s, s, s, k.op, plain(w.Gc[jt][ut + 2 * v], s), R + (size_t)r * s * ld + (size_t)(2 * jt + v) * s,
                           ld, k.alpha, ONE));
    }
    if (nj > 0) {
      const z64* b1 = w.inj;
      const z64* bn = w.inj + (size_t)s * nj;
      const int jl = w.np - 1;
      // gb = g b'': b'_1 sits in slot 0 (partition 0), b'_n in slot NS - 1 (last partition)
      for (int u = 0; u < 2; ++u) {
        gbA.push_back(gdesc(s, nj, s, plain(w.Gc[0][u], s), plain(b1, nj), w.gb + (size_t)u * s * nj, nj, ONE, ZERO));
        gbB.push_back(gdesc(s, nj, s, plain(w.Gc[jl][u + 2], s), plain(bn, nj), w.gb + (size_t)(2 * jl + u) * s * nj, nj,
                            ONE, w.np == 1 ? ONE : ZERO));
      }
      // z right-hand side -K'(r, t) gb(t), non-zero where t is a slot of the first or last partition
      for (int r = 0; r < NS; ++r) {
        const KTerm k = kterm(w, r);
        const int jt = k.t / 2;
        if (jt != 0 && jt != jl) continue;
        gsb.push_back(gdesc(s, nj, s, k.op, plain(w.gb + (size_t)k.t * s * nj, nj), R + (size_t)r * s * ld + S2 + s, ld,
                            zneg(k.alpha), ZERO));
      }
      // c = b'' + z
      for (int r = 0; r < NS; ++r) {
        FormDesc c = fcopy(w.cv + (size_t)r * s * nj, nj, R + (size_t)r * s * ld + S2 + s, ld, s, nj);
        if (r == 0) { c.y = b1; c.ldy = nj; c.ay = ONE; }
        if (r == NS - 1) { c.z = bn; c.ldz = nj; c.az = ONE; }
        fc.push_back(c);
      }
      // x_i = Q^first_i c(2j) + Q^last_i c(2j+1) for block i of partition j
      for (int j = 0; j < w.np; ++j)
        for (int i = w.pa[j]; i <= w.pb[j]; ++i) {
          z64* xi = w.x + (size_t)(i - 1) * s * nj;
          gx1.push_back(gdesc(s, nj, s, plain(w.X[0] + (size_t)(i - 1) * ss2, s),
                              plain(w.cv + (size_t)(2 * j) * s * nj, nj), xi, nj, ONE, ZERO));
          gx2.push_back(gdesc(s, nj, s, plain(w.X[1] + (size_t)(i - 1) * ss2, s),
                              plain(w.cv + (size_t)(2 * j + 1) * s * nj, nj), xi, nj, ONE, ONE));
        }
    }
    LuDesc L{};
    L.w = R; L.ldw = ld; L.s = S2; L.ncols = ld; L.ipiv = w.ipr; L.info = info + p;
    lu.push_back(L);
    // G_1n = g(slot 0, .) R^-1 E_last = G_aa w_0 + G_ab w_1 (w: the E_last solution in partition 0's slots)
    gG1.push_back(gdesc(s, s, s, plain(w.Gc[0][0], s), plain(R + S2, ld), w.G1n, s, ONE, ZERO));
    gG2.push_back(gdesc(s, s, s, plain(w.Gc[0][2], s), plain(R + (size_t)s * ld + S2, ld), w.G1n, s, ONE, ONE));
    // Gamma = i Sigma - i Sigma^H
    for (int q2 = 0; q2 < 2; ++q2) {
      FormDesc gm = fdesc(w.Gam[q2], s, s, s);
      gm.x = w.sig[q2]; gm.ldx = s; gm.ax = make_double2(0.0, 1.0);
      gm.y = w.sig[q2]; gm.ldy = s; gm.ty = 1; gm.ay = make_double2(0.0, -1.0);
      fg.push_back(gm);
    }
    gM.push_back(gdesc(s, s, s, plain(w.Gam[0], s), plain(w.G1n, s), w.M1, s, ONE, ZERO));
    gM.push_back(gdesc(s, s, s, plain(w.Gam[1], s), plain(w.G1n, s, 1), w.M2, s, ONE, ZERO));
    tr.push_back({w.M1, s, w.M2, s, s, traces + p, nullptr});
  }
  B.form(f0);
  big_gemm(h, B, gR);
  big_gemm(h, B, gbA);
  big_gemm(h, B, gbB);
  big_gemm(h, B, gsb);
  ::lu(h, B, lu);
  big_gemm(h, B, gG1);
  big_gemm(h, B, gG2);
  B.form(fc);
  big_gemm(h, B, gx1);
  big_gemm(h, B, gx2);
  B.form(fg);
  big_gemm(h, B, gM);
  B.trace(tr);
}

// ------------------------------------------------------------ refinement
// Residual r = Inj - (A - Sigma) x for every block, and ||r||_F^2 and
// ||x||_F^2.  The products are FP64-accurate (FP64 SIMT, or the exact
// digit-sliced tensor-core GEMM in the mixed mode).
void build_ir_residual(ss_handle* h, std::vector<PW>& pts, int ninj, double* rr, double* xx) {
  Plan& R = h->p_ir_res;
  R.clear();
  const int P = (int)pts.size();
  R.memset0(rr, sizeof(double) * P);
  R.memset0(xx, sizeof(double) * P);
  std::vector<FormDesc> f;
  std::vector<GemmDesc> gd, gu, gl, gs1, gs2;
  std::vector<Norm1Desc> nr;
  for (int p = 0; p < P; ++p) {
    PW& w = pts[p];
    const int n = w.n, s = w.s;
    const size_t ss2 = (size_t)s * s, bs = (size_t)s * ninj;
    const KData* kd = w.kd;
    const z64 E = make_double2(w.E, 0.0);
    for (int i = 1; i <= n; ++i) {
      z64* ri = w.r + (i - 1) * bs;
      FormDesc fd = fdesc(ri, ninj, s, ninj);
      if (i == 1) { fd.x = w.inj; fd.ldx = ninj; fd.ax = ONE; }
      if (i == n) { fd.y = w.inj + bs; fd.ldy = ninj; fd.ay = ONE; }
      f.push_back(fd);
      const z64* xi = w.x + (i - 1) * bs;
      gd.push_back(gdesc(s, ninj, s, formed(kd->Sd + (i - 1) * ss2, kd->Hd + (i - 1) * ss2, E, s), plain(xi, ninj), ri,
                         ninj, MONE, ONE));
      if (i < n)
        gu.push_back(gdesc(s, ninj, s, formed(kd->Su + (i - 1) * ss2, kd->Hu + (i - 1) * ss2, E, s), plain(xi + bs, ninj),
                           ri, ninj, MONE, ONE));
      if (i > 1)
        gl.push_back(gdesc(s, ninj, s, formed(kd->Su + (i - 2) * ss2, kd->Hu + (i - 2) * ss2, E, s, 1),
                           plain(xi - bs, ninj), ri, ninj, MONE, ONE));
    }
    gs1.push_back(gdesc(s, ninj, s, plain(w.sig[0], s), plain(w.x, ninj), w.r, ninj, ONE, ONE));
    gs2.push_back(gdesc(s, ninj, s, plain(w.sig[1], s), plain(w.x + (n - 1) * bs, ninj), w.r + (n - 1) * bs, ninj, ONE,
                        ONE));
    nr.push_back({w.r, ninj, n * s, ninj, rr + p, nullptr});
    nr.push_back({w.x, ninj, n * s, ninj, xx + p, nullptr});
  }
  R.form(f);
  big_gemm(h, R, gd);
  big_gemm(h, R, gu);
  big_gemm(h, R, gl);
  big_gemm(h, R, gs1);
  big_gemm(h, R, gs2);
  R.frob2(nr);
}

// ||A - Sigma||_F^2 of every point (block tridiagonal: diagonal blocks with
// the self-energies on the first and last one, the upper blocks counted
// twice for their conjugate-transposed lower partners) and ||Inj||_F^2.
void build_ir_norms(Plan& N, std::vector<PW>& pts, int ninj, double* mm, double* bb) {
  const int P = (int)pts.size();
  N.memset0(mm, sizeof(double) * P);
  N.memset0(bb, sizeof(double) * P);
  std::vector<FormDesc> f;
  std::vector<Norm1Desc> nb_d;
  for (int p = 0; p < P; ++p) {
    const PW& w = pts[p];
    const int n = w.n, s = w.s;
    const size_t ss2 = (size_t)s * s;
    const KData* kd = w.kd;
    const z64 E = make_double2(w.E, 0.0);
    for (int i = 1; i <= n; ++i) {
      FormDesc d = fformed(nullptr, 0, kd->Sd + (i - 1) * ss2, kd->Hd + (i - 1) * ss2, E, s, s, s);
      if (i == 1) { d.z = w.sig[0]; d.ldz = s; d.az = MONE; }
      if (i == n) { d.v = w.sig[1]; d.ldv = s; d.av = MONE; }
      d.nrm = mm + p; d.nw = 1.0;
      f.push_back(d);
      if (i < n) {
        FormDesc u = fformed(nullptr, 0, kd->Su + (i - 1) * ss2, kd->Hu + (i - 1) * ss2, E, s, s, s);
        u.nrm = mm + p; u.nw = 2.0;
        f.push_back(u);
      }
    }
    nb_d.push_back({w.inj, ninj, 2 * s, ninj, bb + p, nullptr});
  }
  N.form(f);
  N.frob2(nb_d);
}

// Correction delta = M~^-1 r with the stored D_i^-1 (block UL substitution of
// the first-column sweep, inside each partition) and R^-1 (Sherman-Morrison-
// Woodbury with the merged boundary system), then x += delta:
//   y = blockdiag(A_j)^-1 r (UL substitution per partition),
//   delta = y - Q R^-1 K' B^T y.
// FP64-accurate products (the exact tensor-core GEMM): with FP32 ones the
// correction stops contracting on long devices (its error times the condition
// number of A - Sigma nears 1).
void build_ir_correction(ss_handle* h, std::vector<PW>& pts, int ninj, int nsteps) {
  Plan& C = h->p_ir_cor;
  C.clear();
  // backward inside partition [a, b]: w_b = D_b^-1 r_b ; w_i = D_i^-1 (r_i - U_i w_{i+1})
  for (int t = 0; t < nsteps; ++t) {
    std::vector<FormDesc> f;
    std::vector<GemmDesc> g1, g2;
    for (auto& w : pts) {
      const int s = w.s;
      const size_t ss2 = (size_t)s * s, bs = (size_t)s * ninj;
      const z64 E = make_double2(w.E, 0.0);
      for (int j = 0; j < w.np; ++j) {
        const int a = w.pa[j], b = w.pb[j];
        if (t > b - a) continue;
        const int i = b - t;
        z64* ri = w.r + (i - 1) * bs;
        z64* wi = w.wv + (i - 1) * bs;
        z64* tj = w.tv + (size_t)j * bs;  // partition j's scratch
        if (i == b) {
          g2.push_back(gdesc(s, ninj, s, plain(w.Dinv + (i - 1) * ss2, s), plain(ri, ninj), wi, ninj, ONE, ZERO));
        } else {
          f.push_back(fcopy(tj, ninj, ri, ninj, s, ninj));
          g1.push_back(gdesc(s, ninj, s, formed(w.kd->Su + (i - 1) * ss2, w.kd->Hu + (i - 1) * ss2, E, s),
                             plain(wi + bs, ninj), tj, ninj, MONE, ONE));
          g2.push_back(gdesc(s, ninj, s, plain(w.Dinv + (i - 1) * ss2, s), plain(tj, ninj), wi, ninj, ONE, ZERO));
        }
      }
    }
    C.form(f);
    big_gemm(h, C, g1);
    big_gemm(h, C, g2);
  }
  // forward inside the partition: y_a = w_a ; y_i = w_i - D_i^-1 (U_{i-1}^H y_{i-1})  (in place in w)
  for (int t = 1; t < nsteps; ++t) {
    std::vector<GemmDesc> g1, g2;
    for (auto& w : pts) {
      const int s = w.s;
      const size_t ss2 = (size_t)s * s, bs = (size_t)s * ninj;
      const z64 E = make_double2(w.E, 0.0);
      for (int j = 0; j < w.np; ++j) {
        const int a = w.pa[j], b = w.pb[j];
        if (t > b - a) continue;
        const int i = a + t;
        z64* wi = w.wv + (i - 1) * bs;
        z64* tj = w.tv + (size_t)j * bs;
        g1.push_back(gdesc(s, ninj, s, formed(w.kd->Su + (i - 2) * ss2, w.kd->Hu + (i - 2) * ss2, E, s, 1),
                           plain(wi - bs, ninj), tj, ninj, ONE, ZERO));
        g2.push_back(gdesc(s, ninj, s, plain(w.Dinv + (i - 1) * ss2, s), plain(tj, ninj), wi, ninj, MONE, ONE));
      }
    }
    big_gemm(h, C, g1);
    big_gemm(h, C, g2);
  }
  // SMW: zc = -K' B^T y ; z' = R^-1 zc ; x_i += y_i + Q^first_i z'(2j) + Q^last_i z'(2j+1)
  std::vector<GemmDesc> gz, gr, gx1, gx2;
  std::vector<FormDesc> fx;
  for (auto& w : pts) {
    const int s = w.s, S2 = w.rows(), NS = 2 * w.np;
    const size_t ss2 = (size_t)s * s, bs = (size_t)s * ninj;
    const int ld = bound_ld(w, ninj, true);
    for (int r = 0; r < NS; ++r) {
      const KTerm k = kterm(w, r);
      const int blk = (k.t & 1) ? w.pb[k.t / 2] : w.pa[k.t / 2];
      gz.push_back(gdesc(s, ninj, s, k.op, plain(w.wv + (size_t)(blk - 1) * bs, ninj), w.zc + (size_t)r * bs, ninj,
                         zneg(k.alpha), ZERO));
    }
    gr.push_back(gdesc(S2, ninj, S2, plain(w.Rw + S2 + s + ninj, ld), plain(w.zc, ninj), w.tv, ninj, ONE, ZERO));
    for (int j = 0; j < w.np; ++j)
      for (int i = w.pa[j]; i <= w.pb[j]; ++i) {
        z64* xi = w.x + (size_t)(i - 1) * bs;
        FormDesc fd = fcopy(xi, ninj, xi, ninj, s, ninj);
        fd.y = w.wv + (size_t)(i - 1) * bs; fd.ldy = ninj; fd.ay = ONE;
        fx.push_back(fd);
        gx1.push_back(gdesc(s, ninj, s, plain(w.X[0] + (size_t)(i - 1) * ss2, s), plain(w.tv + (size_t)(2 * j) * bs, ninj),
                            xi, ninj, ONE, ONE));
        gx2.push_back(gdesc(s, ninj, s, plain(w.X[1] + (size_t)(i - 1) * ss2, s),
                            plain(w.tv + (size_t)(2 * j + 1) * bs, ninj), xi, ninj, ONE, ONE));
      }
  }
  big_gemm(h, C, gz);
  big_gemm(h, C, gr);
  C.form(fx);
  big_gemm(h, C, gx1);
  big_gemm(h, C, gx2);
}

// ----------------------------------------------------- density of states
// rho_i = -Im Tr[G_ii] / pi for every block of the open system G = (A - Sigma)^-1
// (Eq. negf; the spectral weight the observables of Sec. 2B are built from).
// Two sweeps over M = A - Sigma_L (+) Sigma_R, run together: the backward one
// keeps the right-connected Schur products SR_i = A_{i,i+1} X_{i+1}
// (X_{i+1} = D_{i+1}^-1 A_{i+1,i}), the forward one the left-connected
// SL_i = A_{i,i-1} Y_{i-1}, each in one block column store.  Then
// G_ii = (M_ii - SL_i - SR_i)^-1 for all blocks (batched LUs with identity
// right-hand sides, DOS_ROUND blocks per point at a time) and the trace of
// its diagonal.  The sweeps' last blocks need no factorisation.
void build_dos_sweeps(ss_handle* h, std::vector<PW>& pts, int* info, int nmax) {
  Plan& S = h->p_sweep;
  S.clear();
  const int P = (int)pts.size();
  S.memset0(info, sizeof(int) * 2 * (size_t)P * nmax);
  for (int t = 0; t < nmax; ++t) {
    std::vector<GemmDesc> g;
    std::vector<FormDesc> f, fc;
    std::vector<LuDesc> lu;
    for (int p = 0; p < P; ++p) {
      PW& w = pts[p];
      const int n = w.n, s = w.s;
      if (t >= n) continue;
      const KData* kd = w.kd;
      const size_t ss2 = (size_t)s * s;
      const z64 E = make_double2(w.E, 0.0);
      for (int dir = 0; dir < 2; ++dir) {
        const int i = dir == 0 ? n - t : t + 1;
        z64* store = w.X[dir] + (size_t)(i - 1) * ss2;  // SR_i (dir 0) / SL_i (dir 1)
        if (t > 0) {
          const int up = dir == 0 ? i - 1 : i - 2;
          g.push_back(gdesc(s, s, s, formed(kd->Su + up * ss2, kd->Hu + up * ss2, E, s, dir == 0 ? 0 : 1),
                            plain(w.Xl[0][dir][(t - 1) & 1], s), store, s, ONE, ZERO));
        }
        if (t == n - 1) continue;  // the block the sweep ends on: nothing further needs D_i
        z64* W = w.Ws[0][dir];
        const int ld = 2 * s;
        // D_i = M_ii - (Schur product): the lead term enters at the sweep's first block
        FormDesc d = fformed(W, ld, kd->Sd + (i - 1) * ss2, kd->Hd + (i - 1) * ss2, E, s, s, s);
        if (t > 0) { d.z = store; d.ldz = s; d.az = MONE; }
        if (t == 0) { d.v = w.sig[dir == 0 ? 1 : 0]; d.ldv = s; d.av = MONE; }
        f.push_back(d);
        if (dir == 0) f.push_back(fformed(W + s, ld, kd->Su + (i - 2) * ss2, kd->Hu + (i - 2) * ss2, E, s, s, s, 1));
        else f.push_back(fformed(W + s, ld, kd->Su + (i - 1) * ss2, kd->Hu + (i - 1) * ss2, E, s, s, s, 0));
        LuDesc L{};
        L.w = W; L.ldw = ld; L.s = s; L.ncols = 2 * s; L.ipiv = w.ips[0][dir];
        L.info = info + (size_t)(2 * p + dir) * nmax + t;
        lu.push_back(L);
        fc.push_back(fcopy(w.Xl[0][dir][t & 1], s, W + s, ld, s, s));
      }
    }
    big_gemm(h, S, g);
    S.form(f);
    ::lu(h, S, lu);
    S.form(fc);
  }
}

// Diagonal blocks, DOS_ROUND per point per round: [M_ii - SL_i - SR_i | 1] -> LU
// -> G_ii in the right-hand side -> Tr into traces[p * nmax + i - 1].
void build_dos_diag(ss_handle* h, std::vector<PW>& pts, int* info, z64* traces, int nmax) {
  Plan& B = h->p_bound;
  B.clear();
  const int P = (int)pts.size();
  B.memset0(info, sizeof(int) * (size_t)P * nmax);
  for (int r0 = 0; r0 < nmax; r0 += DOS_ROUND) {
    std::vector<FormDesc> f;
    std::vector<LuDesc> lu;
    std::vector<TraceDesc> tr;
    for (int p = 0; p < P; ++p) {
      PW& w = pts[p];
      const int n = w.n, s = w.s;
      const KData* kd = w.kd;
      const size_t ss2 = (size_t)s * s;
      const z64 E = make_double2(w.E, 0.0);
      for (int q = 0; q < DOS_ROUND; ++q) {
        const int i = r0 + q + 1;
        if (i > n) break;
        z64* K = w.Kw + (size_t)q * 2 * ss2;
        FormDesc d = fformed(K, 2 * s, kd->Sd + (i - 1) * ss2, kd->Hd + (i - 1) * ss2, E, s, s, s);
        // two of: SR_i (i < n), SL_i (i > 1), Sigma_L (i = 1), Sigma_R (i = n)
        const z64* t1 = i < n ? w.X[0] + (size_t)(i - 1) * ss2 : w.sig[1];
        const z64* t2 = i > 1 ? w.X[1] + (size_t)(i - 1) * ss2 : w.sig[0];
        d.z = t1; d.ldz = s; d.az = MONE;
        d.v = t2; d.ldv = s; d.av = MONE;
        f.push_back(d);
        f.push_back(fident(K + s, 2 * s, s, s, 1.0));
        LuDesc L{};
        L.w = K; L.ldw = 2 * s; L.s = s; L.ncols = 2 * s; L.ipiv = w.ipk + (size_t)q * s;
        L.info = info + (size_t)p * nmax + i - 1;
        lu.push_back(L);
        tr.push_back({K + s, 2 * s, nullptr, 0, s, traces + (size_t)p * nmax + i - 1, nullptr});
      }
    }
    B.form(f);
    ::lu(h, B, lu);
    B.trace(tr);
  }
}

// ------------------------------------------- contour-integral (FEAST) leads
// Sec. 3A, Eq. bound and Eq. feast: the lead's Bloch modes psi_q = lambda^q u
// solve (L + lambda D + lambda^2 U) u = 0 (blocks of z S - H at z = E + i eta;
// companion form A v = lambda B v, v = [u; lambda u], A = [[0, 1], [-L, -D]],
// B = [[1, 0], [0, U]]).  Per (point, lead):
//   1. contour solves: X_p = (z_p B - A)^-1 B Y at 2 Np nodes on |z| = R
//      (counterclockwise) and |z| = 1/R (clockwise), Y a fixed 2s x m0 random
//      block; by the block form of z B - A each is one s x s solve,
//      (L + z D + z^2 U) X1 = U (Y2 + z Y1) + D Y1, X2 = z X1 - Y1, all
//      nodes of all problems in one batched LU;
//   2. Q = sum_p (z_p / Np) X_p (minus on the inner circle): the spectral
//      projector onto the annulus 1/R < |lambda| < R applied to Y;
//   3. an orthonormal basis of span Q: eigen-decomposition of the Gram matrix
//      Q^H Q, directions with singular value below 1e-10 of the largest dropped;
//   4. Rayleigh-Ritz: K = (Qt^H B Qt)^-1 (Qt^H A Qt), its eigenpairs (ss_eig.cu),
//      u_j = first half of Qt y_j;
//   5. on the host: the modes inside the annulus going towards the bulk (right
//      lead |lambda| < 1, left lead |lambda| > 1);
//   6. F = U_m diag(f) U_m^+ (f = lambda, or 1/lambda on the left; U_m^+ = U_m^-1
//      when all s modes are found, (U_m^H U_m)^-1 U_m^H otherwise), the surface
//      Green's function g = (D + U F)^-1 (right) or (D + L F)^-1 (left), and
//      Sigma = A_{n,n+1} g A_{n+1,n} / A_{1,0} g A_{0,1} at real E.
struct FeastProb {
  PW* w;
  int q;       // lead: 0 left, 1 right
  int s, m0;   // block size, subspace columns
  int k = 0;   // rank kept after the Gram step
  int mm = 0;  // modes used for F
  // scratch (device)
  z64 *Y, *Wn, *Tn, *Q, *G, *GZ, *GX, *Glam, *Qt, *AQ, *RR, *KZ, *KX, *Klam, *ZX, *Ua, *Ut, *Uf, *PS, *PF, *GG, *F;
  int *piv, *pivn, *info;
};

size_t feast_prob_bytes(int s, int m0, int np2) {
  Carve c(nullptr);
  FeastProb f{};
  f.s = s; f.m0 = m0;
  const size_t sm = (size_t)s * m0, mm2 = (size_t)m0 * m0;
  c.take<z64>(2 * sm); c.take<z64>((size_t)np2 * s * (s + m0)); c.take<z64>((size_t)np2 * sm); c.take<z64>(2 * sm);
  for (int i = 0; i < 3; ++i) c.take<z64>(mm2);
  c.take<z64>(m0); c.take<z64>(2 * sm); c.take<z64>(2 * sm); c.take<z64>((size_t)m0 * 2 * m0);
  for (int i = 0; i < 3; ++i) c.take<z64>(mm2);
  c.take<z64>(m0); c.take<z64>(sm); c.take<z64>(sm); c.take<z64>(sm); c.take<z64>(sm);
  const size_t ps = (size_t)m0 * std::max(m0, s);
  c.take<z64>(ps); c.take<z64>(ps); c.take<z64>((size_t)m0 * (m0 + 2 * s)); c.take<z64>((size_t)s * s);
  c.take<int>((size_t)np2 * s); c.take<int>(2 * m0 + 2 * s);
  return c.off + 256;
}

void feast_carve(Carve& c, FeastProb& f, int np2) {
  const int s = f.s, m0 = f.m0;
  const size_t sm = (size_t)s * m0, mm2 = (size_t)m0 * m0;
  f.Y = c.take<z64>(2 * sm); f.Wn = c.take<z64>((size_t)np2 * s * (s + m0)); f.Tn = c.take<z64>((size_t)np2 * sm);
  f.Q = c.take<z64>(2 * sm);
  f.G = c.take<z64>(mm2); f.GZ = c.take<z64>(mm2); f.GX = c.take<z64>(mm2); f.Glam = c.take<z64>(m0);
  f.Qt = c.take<z64>(2 * sm); f.AQ = c.take<z64>(2 * sm); f.RR = c.take<z64>((size_t)m0 * 2 * m0);
  f.KZ = c.take<z64>(mm2); f.KX = c.take<z64>(mm2); f.ZX = c.take<z64>(mm2); f.Klam = c.take<z64>(m0);
  f.Ua = c.take<z64>(sm); f.Ut = c.take<z64>(sm); f.Uf = c.take<z64>(sm); f.AQ = f.AQ;
  c.take<z64>(sm);
  const size_t ps = (size_t)m0 * std::max(m0, s);
  f.PS = c.take<z64>(ps); f.PF = c.take<z64>(ps); f.GG = c.take<z64>((size_t)m0 * (m0 + 2 * s));
  f.F = c.take<z64>((size_t)s * s);
  f.pivn = c.take<int>((size_t)np2 * s); f.piv = c.take<int>(2 * m0 + 2 * s);
}

// Seeded complex Gaussian-like block (a 64-bit LCG; the subspace only has to
// be generic), the same for every problem of a given shape.
std::vector<z64> feast_random_block(int rows, int cols) {
  std::vector<z64> y((size_t)rows * cols);
  unsigned long long r = 0x9E3779B97F4A7C15ull ^ ((unsigned long long)rows << 32) ^ (unsigned long long)cols;
  for (auto& v : y) {
    r = r * 6364136223846793005ull + 1442695040888963407ull;
    const double a = ((double)((r >> 11) & ((1ull << 52) - 1)) / (double)(1ull << 52)) - 0.5;
    r = r * 6364136223846793005ull + 1442695040888963407ull;
    const double b = ((double)((r >> 11) & ((1ull << 52) - 1)) / (double)(1ull << 52)) - 0.5;
    v = make_double2(a, b);
  }
  return y;
}

z64 zinv_host(z64 a) {
  const double d = a.x * a.x + a.y * a.y;
  return make_double2(a.x / d, -a.y / d);
}

int run_feast(ss_handle* h, std::vector<PW>& pts) {
  cudaStream_t st = h->stream;
  const int P = (int)pts.size();
  const int np = h->cfg.feast_points;
  const int np2 = 2 * np;
  const double Rr = h->cfg.feast_radius, eta = h->cfg.eta;
  std::vector<FeastProb> fp;
  size_t bytes = 0;
  for (auto& w : pts)
    for (int q = 0; q < 2; ++q) {
      FeastProb f{};
      f.w = &w; f.q = q; f.s = w.s;
      f.m0 = h->cfg.feast_subspace > 0 ? std::min(h->cfg.feast_subspace, 2 * w.s) : 2 * w.s;
      bytes += feast_prob_bytes(f.s, f.m0, np2);
      fp.push_back(f);
    }
  if (bytes > h->feast_bytes) {
    cudaFree(h->feast_buf);
    h->feast_buf = nullptr; h->feast_bytes = 0;
    CK(cudaMalloc(&h->feast_buf, bytes), "contour-integral scratch");
    h->feast_bytes = bytes;
  }
  Carve c(h->feast_buf);
  for (auto& f : fp) feast_carve(c, f, np2);
  if (h->feast_info_n < 8 * fp.size()) {
    cudaFree(h->feast_info);
    h->feast_info = nullptr; h->feast_info_n = 0;
    CK(cudaMalloc(&h->feast_info, sizeof(int) * 8 * fp.size()), "contour-integral flags");
    h->feast_info_n = 8 * fp.size();
  }
  for (size_t i = 0; i < fp.size(); ++i) fp[i].info = h->feast_info + 8 * i;
  // random blocks Y (host, uploaded)
  for (auto& f : fp) {
    const std::vector<z64> y = feast_random_block(2 * f.s, f.m0);
    CK(cudaMemcpyAsync(f.Y, y.data(), y.size() * sizeof(z64), cudaMemcpyHostToDevice, st), "feast Y");
  }
  // ---------------- plan A: lead blocks, contour solves, Q, Gram matrix, its eigenpairs
  Plan& A = h->p_fa;
  A.clear();
  {
    std::vector<FormDesc> f0, f1;
    std::vector<std::vector<FormDesc>> qpass;  // per problem: the running-sum passes, then the Y1 term
    std::vector<GemmDesc> g1, g2, gG, gG2;
    std::vector<LuDesc> lu;
    std::vector<EigDesc> eg;
    for (auto& f : fp) {
      PW& w = *f.w;
      const int s = f.s, m0 = f.m0, q = f.q;
      const z64 z = make_double2(w.E, eta);
      const z64* const* cc = w.kd->cell[q];
      z64 *D = w.D[q], *U = w.a[q][0], *L = w.b[q][0];
      f0.push_back(fformed(D, s, cc[2], cc[0], z, s, s, s));
      f0.push_back(fformed(U, s, cc[3], cc[1], z, s, s, s));
      f0.push_back(fformed(L, s, cc[3], cc[1], z, s, s, s, 1));
      const z64* Y1 = f.Y;
      const z64* Y2 = f.Y + (size_t)s * m0;
      for (int p = 0; p < np2; ++p) {
        const bool outer = p < np;
        const double rad = outer ? Rr : 1.0 / Rr, th = 2.0 * M_PI * ((p % np) + 0.5) / np;
        const z64 zp = make_double2(rad * std::cos(th), rad * std::sin(th));
        const z64 zp2 = zmul(zp, zp);
        z64* W = f.Wn + (size_t)p * s * (s + m0);
        const int ld = s + m0;
        // P(z) = L + z D + z^2 U
        FormDesc pz = fdesc(W, ld, s, s);
        pz.x = L; pz.ldx = s; pz.ax = ONE;
        pz.y = D; pz.ldy = s; pz.ay = zp;
        pz.z = U; pz.ldz = s; pz.az = zp2;
        f1.push_back(pz);
        // T = Y2 + z Y1 ; rhs = U T + D Y1
        z64* T = f.Tn + (size_t)p * s * m0;
        FormDesc tf = fdesc(T, m0, s, m0);
        tf.x = Y2; tf.ldx = m0; tf.ax = ONE;
        tf.y = Y1; tf.ldy = m0; tf.ay = zp;
        f1.push_back(tf);
        g1.push_back(gdesc(s, m0, s, plain(U, s), plain(T, m0), W + s, ld, ONE, ZERO));
        g2.push_back(gdesc(s, m0, s, plain(D, s), plain(Y1, m0), W + s, ld, ONE, ONE));
        LuDesc Ld{};
        Ld.w = W; Ld.ldw = ld; Ld.s = s; Ld.ncols = s + m0; Ld.ipiv = f.pivn + (size_t)p * s; Ld.info = f.info;
        lu.push_back(Ld);
      }
      // Q1 = sum_p c_p X1_p, Q2 = sum_p c_p (z_p X1_p - Y1): c_p = +z_p / Np outer,
      // -z_p / Np inner; three nodes per form pass (terms x, y, z; v carries the
      // running sum), passes of one problem in consecutive launches
      z64* Q1 = f.Q;
      z64* Q2 = f.Q + (size_t)s * m0;
      z64 csum = ZERO;
      std::vector<FormDesc> mine;
      for (int p0 = 0; p0 < np2; p0 += 3) {
        FormDesc a1 = fdesc(Q1, m0, s, m0), a2 = fdesc(Q2, m0, s, m0);
        const z64* src[3] = {nullptr, nullptr, nullptr};
        z64 co[3], co2[3];
        for (int t = 0; t < 3; ++t) {
          const int p = p0 + t;
          if (p >= np2) break;
          const bool outer = p < np;
          const double rad = outer ? Rr : 1.0 / Rr, th = 2.0 * M_PI * ((p % np) + 0.5) / np;
          const z64 zp = make_double2(rad * std::cos(th), rad * std::sin(th));
          const z64 cp = make_double2((outer ? 1.0 : -1.0) * zp.x / np, (outer ? 1.0 : -1.0) * zp.y / np);
          src[t] = f.Wn + (size_t)p * s * (s + m0) + s;
          co[t] = cp;
          co2[t] = zmul(cp, zp);
          csum = zadd(csum, cp);
        }
        a1.x = src[0]; a1.ldx = s + m0; a1.ax = co[0];
        a2.x = src[0]; a2.ldx = s + m0; a2.ax = co2[0];
        if (src[1]) { a1.y = src[1]; a1.ldy = s + m0; a1.ay = co[1]; a2.y = src[1]; a2.ldy = s + m0; a2.ay = co2[1]; }
        if (src[2]) { a1.z = src[2]; a1.ldz = s + m0; a1.az = co[2]; a2.z = src[2]; a2.ldz = s + m0; a2.az = co2[2]; }
        if (p0 > 0) { a1.v = Q1; a1.ldv = m0; a1.av = ONE; a2.v = Q2; a2.ldv = m0; a2.av = ONE; }
        mine.push_back(a1);
        mine.push_back(a2);
      }
      // the -Y1 terms of Q2: - (sum_p c_p) Y1
      FormDesc fy = fcopy(Q2, m0, Q2, m0, s, m0);
      fy.y = Y1; fy.ldy = m0; fy.ay = make_double2(-csum.x, -csum.y);
      mine.push_back(fy);
      qpass.push_back(mine);
      // Gram matrix Q^H Q = Q1^H Q1 + Q2^H Q2 (two launches: both write G)
      gG.push_back(gdesc(m0, m0, s, plain(Q1, m0, 1), plain(Q1, m0), f.G, m0, ONE, ZERO));
      gG2.push_back(gdesc(m0, m0, s, plain(Q2, m0, 1), plain(Q2, m0), f.G, m0, ONE, ONE));
      eg.push_back({f.G, f.GZ, f.GX, f.Glam, m0, m0, f.info + 1});
    }
    A.memset0(h->feast_info, sizeof(int) * h->feast_info_n);
    A.form(f0);
    A.form(f1);
    A.gemm(g1);
    A.gemm(g2);
    ::lu(h, A, lu);
    // the passes of one problem are sequential (running sums): one launch per pass index
    const size_t npass = qpass.empty() ? 0 : qpass[0].size();
    for (size_t k = 0; k + 1 < npass; k += 2) {
      std::vector<FormDesc> one;
      for (auto& v : qpass) { one.push_back(v[k]); one.push_back(v[k + 1]); }
      A.form(one);
    }
    std::vector<FormDesc> last;
    for (auto& v : qpass) last.push_back(v.back());
    A.form(last);
    A.gemm(gG);
    A.gemm(gG2);
    A.eig(eg);
  }
  CK(A.upload(st), "upload feast A");
  CK(A.run(st, &h->nlaunch, h->P()), "feast contour solves");
  // ---------------- host: rank of Q from the Gram eigenvalues
  std::vector<std::vector<z64>> glam(fp.size());
  for (size_t i = 0; i < fp.size(); ++i) {
    glam[i].resize(fp[i].m0);
    CK(cudaMemcpyAsync(glam[i].data(), fp[i].Glam, sizeof(z64) * fp[i].m0, cudaMemcpyDeviceToHost, st), "gram");
  }
  std::vector<int> finfo(h->feast_info_n);
  CK(cudaMemcpyAsync(finfo.data(), h->feast_info, sizeof(int) * finfo.size(), cudaMemcpyDeviceToHost, st), "info");
  CK(cudaStreamSynchronize(st), "feast sync");
  for (size_t i = 0; i < fp.size(); ++i) {
    FeastProb& f = fp[i];
    if (finfo[(i * 8)] || finfo[i * 8 + 1]) return fail(h, SS_ERR_SINGULAR, "contour-integral solve failed (singular node or eigen-iteration cap)");
    double mx = 0.0;
    for (auto& v : glam[i]) mx = std::max(mx, v.x);
    std::vector<z64> S((size_t)f.m0 * f.m0, ZERO);
    int k = 0;
    for (int j = 0; j < f.m0; ++j)
      if (glam[i][j].x > 1e-20 * mx) { S[(size_t)j * f.m0 + k] = make_double2(1.0 / std::sqrt(glam[i][j].x), 0.0); ++k; }
    f.k = k;
    CK(cudaMemcpyAsync(f.PS, S.data(), S.size() * sizeof(z64), cudaMemcpyHostToDevice, st), "scaling");
  }
  // ---------------- plan B: orthonormal basis, Rayleigh-Ritz, eigenpairs of K
  Plan& B = h->p_fb;
  B.clear();
  {
    std::vector<GemmDesc> gV, gQ, gA1, gA2, gR1, gR2, gR3, gR4;
    std::vector<LuDesc> lu;
    std::vector<EigDesc> eg;
    for (auto& f : fp) {
      PW& w = *f.w;
      const int s = f.s, m0 = f.m0, k = f.k, q = f.q;
      z64 *D = w.D[q], *U = w.a[q][0], *L = w.b[q][0];
      // Vs = GZ * PS (m0 x k), Qt = Q Vs (2s x k): orthonormal basis of span Q
      gV.push_back(gdesc(m0, k, m0, plain(f.GZ, m0), plain(f.PS, m0), f.GX, k, ONE, ZERO));
      gQ.push_back(gdesc(2 * s, k, m0, plain(f.Q, m0), plain(f.GX, k), f.Qt, k, ONE, ZERO));
      const z64* Qt1 = f.Qt;
      const z64* Qt2 = f.Qt + (size_t)s * k;
      // A Qt = [Qt2; -L Qt1 - D Qt2], B Qt = [Qt1; U Qt2]
      z64* AQ2 = f.AQ;
      z64* BQ2 = f.AQ + (size_t)s * k;
      gA1.push_back(gdesc(s, k, s, plain(L, s), plain(Qt1, k), AQ2, k, MONE, ZERO));
      gA2.push_back(gdesc(s, k, s, plain(D, s), plain(Qt2, k), AQ2, k, MONE, ONE));
      gA1.push_back(gdesc(s, k, s, plain(U, s), plain(Qt2, k), BQ2, k, ONE, ZERO));
      // RR = [Qt^H B Qt | Qt^H A Qt] (k x 2k)
      z64* Bh = f.RR;
      z64* Ah = f.RR + k;
      gR1.push_back(gdesc(k, k, s, plain(Qt1, k, 1), plain(Qt1, k), Bh, 2 * k, ONE, ZERO));
      gR2.push_back(gdesc(k, k, s, plain(Qt2, k, 1), plain(BQ2, k), Bh, 2 * k, ONE, ONE));
      gR3.push_back(gdesc(k, k, s, plain(Qt1, k, 1), plain(Qt2, k), Ah, 2 * k, ONE, ZERO));
      gR4.push_back(gdesc(k, k, s, plain(Qt2, k, 1), plain(AQ2, k), Ah, 2 * k, ONE, ONE));
      LuDesc Ld{};
      Ld.w = f.RR; Ld.ldw = 2 * k; Ld.s = k; Ld.ncols = 2 * k; Ld.ipiv = f.piv; Ld.info = f.info + 2;
      lu.push_back(Ld);
    }
    B.gemm(gV);
    B.gemm(gQ);
    B.gemm(gA1);
    B.gemm(gA2);
    B.gemm(gR1);
    B.gemm(gR2);
    B.gemm(gR3);
    B.gemm(gR4);
    ::lu(h, B, lu);
    // K = B^-1 A sits in the right half of RR: copy it out (ld k) for the eigen-solver
    std::vector<FormDesc> fk;
    for (auto& f : fp) {
      fk.push_back(fcopy(f.KZ, f.k, f.RR + f.k, 2 * f.k, f.k, f.k));
      eg.push_back({f.KZ, f.KX, f.ZX, f.Klam, f.k, f.k, f.info + 3});
    }
    B.form(fk);
    B.eig(eg);
    // eigenvectors of K: (Z X); modes u = first half of Qt (Z X)
    std::vector<GemmDesc> gY, gU;
    for (auto& f : fp) {
      const int s = f.s, k = f.k;
      gY.push_back(gdesc(k, k, k, plain(f.KX, k), plain(f.ZX, k), f.GX, k, ONE, ZERO));
      gU.push_back(gdesc(s, k, k, plain(f.Qt, k), plain(f.GX, k), f.Ua, k, ONE, ZERO));
    }
    B.gemm(gY);
    B.gemm(gU);
  }
  CK(B.upload(st), "upload feast B");
  CK(B.run(st, &h->nlaunch, h->P()), "feast Rayleigh-Ritz");
  std::vector<std::vector<z64>> lam(fp.size());
  for (size_t i = 0; i < fp.size(); ++i) {
    lam[i].resize(fp[i].k);
    CK(cudaMemcpyAsync(lam[i].data(), fp[i].Klam, sizeof(z64) * fp[i].k, cudaMemcpyDeviceToHost, st), "ritz values");
  }
  CK(cudaMemcpyAsync(finfo.data(), h->feast_info, sizeof(int) * finfo.size(), cudaMemcpyDeviceToHost, st), "info");
  CK(cudaStreamSynchronize(st), "feast sync");
  // ---------------- host: modes inside the annulus moving towards the bulk
  for (size_t i = 0; i < fp.size(); ++i) {
    FeastProb& f = fp[i];
    if (finfo[i * 8 + 2] || finfo[i * 8 + 3])
      return fail(h, SS_ERR_SINGULAR, "contour-integral Rayleigh-Ritz failed (singular B^ or eigen-iteration cap)");
    std::vector<z64> S((size_t)f.k * f.s, ZERO), Sf((size_t)f.k * f.s, ZERO);
    int m = 0;
    for (int j = 0; j < f.k && m < f.s; ++j) {
      const double a = std::hypot(lam[i][j].x, lam[i][j].y);
      if (!(a > 1.0 / Rr && a < Rr)) continue;
      if (f.q == 1 ? !(a < 1.0) : !(a > 1.0)) continue;
      const z64 l = lam[i][j];
      const z64 fv = f.q == 1 ? l : zinv_host(l);
      S[(size_t)j * f.s + m] = ONE;  // column m of U_m = column j of Ua (k x s selection, ld s)
      Sf[(size_t)j * f.s + m] = fv;
      ++m;
    }
    f.mm = m;
    if (m == 0) return fail(h, SS_ERR_SINGULAR, "no lead mode found inside the annulus");
    CK(cudaMemcpyAsync(f.PS, S.data(), S.size() * sizeof(z64), cudaMemcpyHostToDevice, st), "selection");
    CK(cudaMemcpyAsync(f.PF, Sf.data(), Sf.size() * sizeof(z64), cudaMemcpyHostToDevice, st), "selection");
  }
  // ---------------- plan C: F, surface Green's function, self-energy
  Plan& C = h->p_fc;
  C.clear();
  {
    std::vector<GemmDesc> gS, gG1, gF, gE, gSig;
    std::vector<FormDesc> fU, fE, fT, fS;
    std::vector<LuDesc> lu1, lu2;
    for (auto& f : fp) {
      PW& w = *f.w;
      const int s = f.s, k = f.k, m = f.mm, q = f.q;
      z64 *D = w.D[q], *U = w.a[q][0], *L = w.b[q][0];
      // Ut = Ua Psel (s x m), Uf = Ua Pf (s x m)
      gS.push_back(gdesc(s, m, k, plain(f.Ua, k), plain(f.PS, s), f.Ut, m, ONE, ZERO));
      gS.push_back(gdesc(s, m, k, plain(f.Ua, k), plain(f.PF, s), f.Uf, m, ONE, ZERO));
      // GG = [Ut^H Ut | Ut^H] (m x (m + s)) -> (Ut^H Ut)^-1 Ut^H, or for m = s [Ut^H | Uf^H] -> Ut^-H Uf^H = F^H
      if (m == s) {
        fU.push_back(fcopy(f.GG, 2 * s, f.Ut, s, s, s, 1));
        fU.push_back(fcopy(f.GG + s, 2 * s, f.Uf, s, s, s, 1));
        LuDesc Ld{};
        Ld.w = f.GG; Ld.ldw = 2 * s; Ld.s = s; Ld.ncols = 2 * s; Ld.ipiv = f.piv; Ld.info = f.info + 4;
        lu1.push_back(Ld);
        fT.push_back(fcopy(f.F, s, f.GG + s, 2 * s, s, s, 1));  // F = (F^H)^H
      } else {
        gG1.push_back(gdesc(m, m, s, plain(f.Ut, m, 1), plain(f.Ut, m), f.GG, m + s, ONE, ZERO));
        fU.push_back(fcopy(f.GG + m, m + s, f.Ut, m, m, s, 1));
        LuDesc Ld{};
        Ld.w = f.GG; Ld.ldw = m + s; Ld.s = m; Ld.ncols = m + s; Ld.ipiv = f.piv; Ld.info = f.info + 4;
        lu1.push_back(Ld);
        gF.push_back(gdesc(s, s, m, plain(f.Uf, m), plain(f.GG + m, m + s), f.F, s, ONE, ZERO));
      }
      // es = D + U F (right) / D + L F (left) into Wd = [es | A]
      const z64 E = make_double2(w.E, 0.0);
      const z64* const* cc = w.kd->cell[q];
      z64* W = w.Wd[q];
      const int ld = 3 * s;
      fE.push_back(fcopy(W, ld, D, s, s, s));
      gE.push_back(gdesc(s, s, s, plain(q == 1 ? U : L, s), plain(f.F, s), W, ld, ONE, ONE));
      // right: rhs A_{n+1,n} = (E S01 - H01)^H ; left: rhs A_{0,1} = E S01 - H01
      fS.push_back(fformed(W + s, ld, cc[3], cc[1], E, s, s, s, q == 1 ? 1 : 0));
      LuDesc L2{};
      L2.w = W; L2.ldw = ld; L2.s = s; L2.ncols = 2 * s; L2.ipiv = w.ipd[q]; L2.info = f.info + 5;
      lu2.push_back(L2);
      gSig.push_back(gdesc(s, s, s, formed(cc[3], cc[1], E, s, q == 1 ? 0 : 1), plain(W + s, ld), w.sig[q], s, ONE, ZERO));
    }
    C.gemm(gS);
    C.gemm(gG1);
    C.form(fU);
    ::lu(h, C, lu1);
    C.gemm(gF);
    C.form(fT);
    C.form(fE);
    C.gemm(gE);
    C.form(fS);
    ::lu(h, C, lu2);
    C.gemm(gSig);
  }
  if (h->plan_error) return fail(h, SS_ERR_OOM, "tensor-core packing buffer too small for the contour solver");
  CK(C.upload(st), "upload feast C");
  CK(C.run(st, &h->nlaunch, h->P()), "feast self-energy");
  CK(cudaMemcpyAsync(finfo.data(), h->feast_info, sizeof(int) * finfo.size(), cudaMemcpyDeviceToHost, st), "info");
  CK(cudaStreamSynchronize(st), "feast sync");
  for (size_t i = 0; i < fp.size(); ++i)
    if (finfo[i * 8 + 4] || finfo[i * 8 + 5]) return fail(h, SS_ERR_SINGULAR, "singular mode matrix or surface block");
  return SS_OK;
}

bool same_points(const ss_handle* h, int n, const double* E, const int* k) {
  if ((int)h->cE.size() != n) return false;
  for (int i = 0; i < n; ++i)
    if (h->cE[i] != E[i] || h->cK[i] != k[i]) return false;
  return true;
}

int ensure_scalars(ss_handle* h, size_t ni, size_t nd, size_t nt) {
  if (ni > h->dint_n) {
    cudaFree(h->dint); h->dint = nullptr; h->dint_n = 0;
    CK(cudaMalloc(&h->dint, ni * sizeof(int)), "cudaMalloc(flags)");
    h->dint_n = ni;
  }
  if (nd > h->ddbl_n) {
    cudaFree(h->ddbl); h->ddbl = nullptr; h->ddbl_n = 0;
    CK(cudaMalloc(&h->ddbl, nd * sizeof(double)), "cudaMalloc(norms)");
    h->ddbl_n = nd;
  }
  if (nt > h->dtr_n) {
    cudaFree(h->dtr); h->dtr = nullptr; h->dtr_n = 0;
    CK(cudaMalloc(&h->dtr, nt * sizeof(z64)), "cudaMalloc(traces)");
    h->dtr_n = nt;
  }
  return SS_OK;
}

// What a pipeline call must produce.
struct Want {
  bool sigma_out = false;
  bool solve = false;   // sweeps + boundary + trace
  bool dos = false;     // density of states per block (instead of solve)
  int ninj = 0;
  const ss_c64* inj = nullptr;
  ss_c64* x = nullptr;
  ss_c64* sigL = nullptr;
  ss_c64* sigR = nullptr;
  double* dos_out = nullptr;
  Layout layout() const { return dos ? LAYOUT_DOS : (solve && !x ? LAYOUT_LEAN : LAYOUT_FULL); }
};

int worst(int a, int b) { return a != SS_OK ? a : b; }

// Run the pipeline over the points of one call (chunked).
int run_points(ss_handle* h, int n_pts, const double* E, const int* k_id, const Want& want,
               std::vector<int>& status, std::vector<int>& iters, std::vector<double>& T,
               std::vector<double>& Ti) {
  if (n_pts < 0) return fail(h, SS_ERR_ARG, "n_pts < 0");
  if (n_pts == 0) return SS_OK;
  if (!E || !k_id) return fail(h, SS_ERR_ARG, "E and k_id must be non-NULL");
  if (want.ninj < 0 || want.ninj > h->cfg.max_inj) return fail(h, SS_ERR_ARG, "n_inj outside 1..max_inj");
  status.assign(n_pts, SS_OK);
  iters.assign(2 * n_pts, 0);
  std::vector<double> err_out(n_pts, -1.0);
  T.assign(n_pts, 0.0);
  Ti.assign(n_pts, 0.0);
  // offsets of per-point packed arrays
  std::vector<size_t> off_ss(n_pts), off_inj(n_pts), off_x(n_pts), off_n(n_pts);
  size_t a_ss = 0, a_inj = 0, a_x = 0, a_n = 0;
  std::vector<int> order(n_pts);
  for (int i = 0; i < n_pts; ++i) {
    auto it = h->ks.find(k_id[i]);
    if (it == h->ks.end()) return fail(h, SS_ERR_STATE, "no Hamiltonian set for k_id " + std::to_string(k_id[i]));
    if (!std::isfinite(E[i])) return fail(h, SS_ERR_ARG, "non-finite energy");
    const int s = it->second.s, n = it->second.n;
    off_ss[i] = a_ss; a_ss += (size_t)s * s;
    off_inj[i] = a_inj; a_inj += (size_t)2 * s * want.ninj;
    off_x[i] = a_x; a_x += (size_t)n * s * want.ninj;
    off_n[i] = a_n; a_n += (size_t)n;
    order[i] = i;
  }
  // longest-processing-time first
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const KData& ka = h->ks[k_id[a]];
    const KData& kb = h->ks[k_id[b]];
    return (double)ka.n * ka.s * ka.s * ka.s > (double)kb.n * kb.s * kb.s * kb.s;
  });
  const bool dp = h->cfg.device_ptrs != 0;
  cudaStream_t st = h->stream;
  int rc_all = SS_OK;
  const Layout layout = want.layout();
  const int parts = layout == LAYOUT_DOS ? 1 : h->cfg.partitions;
  // reuse of the previous call's self-energies when the point list is
  // identical and, in this call's layout too, forms one batch (the doubling
  // buffers then sit at the same addresses)
  bool one_batch = n_pts <= h->cfg.max_points;
  {
    size_t tot = 0;
    for (int i = 0; i < n_pts && one_batch; ++i) {
      const KData& kd = h->ks[k_id[i]];
      tot += point_bytes(kd.n, kd.s, h->cfg.max_inj, h->mixed(), layout, parts);
    }
    one_batch = one_batch && tot <= h->arena_bytes;
  }
  const bool reuse_sigma = h->c_sigma && same_points(h, n_pts, E, k_id) && one_batch;
  // the first-column sweep keeps D_i^-1 only when x is refined
  const bool refine = h->mixed() && layout == LAYOUT_FULL && want.x && want.ninj > 0;

  size_t pos = 0;
  while (pos < (size_t)n_pts) {
    // chunk: as many points as fit the arena and max_points
    std::vector<PW> pts;
    size_t bytes = 0;
    while (pos < (size_t)n_pts && (int)pts.size() < h->cfg.max_points) {
      const int i = order[pos];
      const KData& kd = h->ks[k_id[i]];
      const size_t need = point_bytes(kd.n, kd.s, h->cfg.max_inj, h->mixed(), layout, parts);
      if (!pts.empty() && bytes + need > h->arena_bytes) break;
      if (need > h->arena_bytes) return fail(h, SS_ERR_OOM, "one point does not fit the workspace");
      bytes += need;
      PW w;
      w.idx = i; w.n = kd.n; w.s = kd.s; w.E = E[i]; w.kd = &kd; w.layout = layout;
      set_partitions(w, parts);
      pts.push_back(w);
      ++pos;
    }
    const int P = (int)pts.size();
    // the layout depends only on (n, s) and max_inj, so cached self-energies
    // stay at the same addresses whatever n_inj the next call uses
    Carve c(h->arena);
    carve_batch(c, pts, h->cfg.max_inj, h->mixed());
    int nmax = 0, smax_c = 0;
    for (auto& w : pts) { nmax = std::max(nmax, w.n); smax_c = std::max(smax_c, w.s); }
    {
      // FP64 GEMM tile shapes tuned for the batch's largest block size
      auto tt = h->tune.find(smax_c);
      const int gsq = tt != h->tune.end() ? tt->second.gsq : -1, gup = tt != h->tune.end() ? tt->second.gup : -1;
      for (Plan* pl : {&h->p_setup, &h->p_iter[0], &h->p_iter[1], &h->p_final, &h->p_sweep, &h->p_bound, &h->p_ir_res,
                       &h->p_ir_cor})
        pl->set_gemm_variants(gsq, gup);
    }
    const int nsteps = sweep_steps(pts);
    // device scalars: act, iters, conv (2P each), decim info (4P), sweep info
    // (2 MAXP P nsteps), boundary / density-of-states info (P nmax)
    const size_t n_sinfo = 2 * (size_t)MAXP * P * std::max(nsteps, 1);
    const size_t ni = 2 * P * 3 + 4 * P + n_sinfo + (size_t)P * nmax;
    int rc = ensure_scalars(h, ni, 3 * 2 * P + 4 * P + (size_t)P * nmax, (size_t)P * nmax);
    if (rc) return rc;
    int* act = h->dint;
    int* itr = act + 2 * P;
    int* conv = itr + 2 * P;
    int* dinfo = conv + 2 * P;
    int* sinfo = dinfo + 4 * P;
    int* binfo = sinfo + n_sinfo;
    double* na = h->ddbl;
    double* nb = na + 2 * P;
    double* nd = nb + 2 * P;
    double* rr = nd + 2 * P;  // refinement: ||r||^2, ||Inj||^2, ||A - Sigma||^2, ||x||^2 per point
    double* bb = rr + P;
    double* mm = bb + P;
    double* xx = mm + P;
    double* dosv = xx + P;    // density of states, P x nmax

    // inputs
    if (want.solve && want.ninj > 0 && layout == LAYOUT_FULL) {
      for (auto& w : pts) {
        const size_t cnt = (size_t)2 * w.s * want.ninj;
        const ss_c64* src = want.inj + off_inj[w.idx];
        if (dp) CK(cudaMemcpyAsync(w.inj, src, cnt * sizeof(z64), cudaMemcpyDeviceToDevice, st), "copy inj");
        else CK(cudaMemcpyAsync(w.inj, src, cnt * sizeof(z64), cudaMemcpyHostToDevice, st), "copy inj");
        if (dp && want.x) w.x = reinterpret_cast<z64*>(want.x + off_x[w.idx]);
      }
    }

    // 1. self-energies
    std::vector<int> h_it(2 * P, 0), h_conv(2 * P, 1), h_dinfo(4 * P, 0);
    std::vector<int> seeded;  // 2 per point: lead seeded by an accepted warm start
    if (!reuse_sigma) {
      h->plan_error = false;
      if (h->cfg.obc == SS_OBC_FEAST) {
        // the leads' Bloch modes by the contour integral, then Sigma from them
        const int r = run_feast(h, pts);
        if (r) {
          for (auto& w : pts) status[w.idx] = r;
          return r;
        }
      } else {
      if (h->cfg.warm_start) {
        // learned warm start of each lead that has a network attached (points
        // of the network's block size); rejected seeds fall back to the doubling
        seeded.assign(2 * P, 0);
        for (int side = 0; side < 2; ++side) {
          if (!h->warm_net[side]) continue;
          int n_in = 0, n_out = 0, mb = 0;
          mlp_dims(h->warm_net[side], &n_in, &n_out, &mb);
          std::vector<PW> sub;
          std::vector<int> where;
          std::vector<double> kv;
          for (int p = 0; p < P; ++p)
            if (2 * pts[p].s * pts[p].s == n_out) { sub.push_back(pts[p]); where.push_back(p); kv.push_back(pts[p].kd->kval); }
          if (sub.empty()) continue;
          std::vector<int> acc;
          const int r = warm_seed(h, sub, side, kv, WARM_ITERS, WARM_TOL, dinfo, acc);
          if (r) return r;
          for (size_t q = 0; q < sub.size(); ++q) seeded[2 * where[q] + side] = acc[q];
        }
      }
      const bool preset = !seeded.empty();
      build_decimation(h, pts, act, itr, conv, dinfo, na, nb, nd, preset, preset ? &seeded : nullptr);
      if (h->plan_error) return fail(h, SS_ERR_OOM, "tensor-core packing buffer too small for the doubling");
      if (preset) {
        std::vector<int> init(2 * P);
        for (int i = 0; i < 2 * P; ++i) init[i] = seeded[i] ? 0 : 1;
        CK(cudaMemcpyAsync(act, init.data(), sizeof(int) * 2 * P, cudaMemcpyHostToDevice, st), "flags");
        CK(cudaStreamSynchronize(st), "flags");
      }
      CK(h->p_setup.upload(st), "upload setup");
      CK(h->p_iter[0].upload(st), "upload iter");
      CK(h->p_iter[1].upload(st), "upload iter");
      CK(h->p_final.upload(st), "upload final");
      CK(h->p_setup.execute(st, &h->nlaunch, h->P(), h->cfg.use_graphs), "decimation setup");
      std::vector<int> h_act(2 * P, 1);
      const int cap = h->cfg.decim_max_iter;
      if (h->cfg.profile) {
        // one step at a time so the flop count sees exactly the active problems
        h->prof.act_dev = act;
        h->prof.act_host = h_act.data();
        h->prof.nact = 2 * P;
        CK(cudaMemcpyAsync(h_act.data(), act, sizeof(int) * 2 * P, cudaMemcpyDeviceToHost, st), "read flags");
        CK(cudaStreamSynchronize(st), "doubling sync");
        for (int it = 0; it < cap + 1; ++it) {
          bool any = false;
          for (int v : h_act) any = any || v;
          if (!any) break;
          CK(h->p_iter[it & 1].run(st, &h->nlaunch, &h->prof), "doubling step");
          CK(cudaMemcpyAsync(h_act.data(), act, sizeof(int) * 2 * P, cudaMemcpyDeviceToHost, st), "read flags");
          CK(cudaStreamSynchronize(st), "doubling sync");
        }
        h->prof.act_host = nullptr;
        h->prof.collect();
      } else {
        for (int it = 0; it < cap + 2; it += 2) {
          if (h->cfg.use_graphs) {
            CK(h->p_iter[0].replay(st, &h->nlaunch), "doubling step");
            CK(h->p_iter[1].replay(st, &h->nlaunch), "doubling step");
          } else {
            CK(h->p_iter[0].run(st, &h->nlaunch), "doubling step");
            CK(h->p_iter[1].run(st, &h->nlaunch), "doubling step");
          }
          CK(cudaMemcpyAsync(h_act.data(), act, sizeof(int) * 2 * P, cudaMemcpyDeviceToHost, st), "read flags");
          CK(cudaStreamSynchronize(st), "doubling sync");
          bool any = false;
          for (int v : h_act) any = any || v;
          if (!any) break;
        }
      }
      CK(h->p_final.execute(st, &h->nlaunch, h->P(), h->cfg.use_graphs), "self-energy");
      CK(cudaMemcpyAsync(h_it.data(), itr, sizeof(int) * 2 * P, cudaMemcpyDeviceToHost, st), "read iters");
      CK(cudaMemcpyAsync(h_conv.data(), conv, sizeof(int) * 2 * P, cudaMemcpyDeviceToHost, st), "read conv");
      CK(cudaMemcpyAsync(h_dinfo.data(), dinfo, sizeof(int) * 4 * P, cudaMemcpyDeviceToHost, st), "read info");
      CK(cudaStreamSynchronize(st), "self-energy sync");
      for (int i = 0; i < (int)seeded.size(); ++i)
        if (seeded[i]) { h_conv[i] = 1; h_it[i] = -WARM_ITERS; }  // accepted seed: converged, steps as negative count
      }

    } else {
      for (int p = 0; p < P; ++p) {
        h_it[2 * p] = h->c_iters[2 * pts[p].idx];
        h_it[2 * p + 1] = h->c_iters[2 * pts[p].idx + 1];
      }
    }
    if (want.sigma_out) {
      for (auto& w : pts) {
        const size_t cnt = (size_t)w.s * w.s * sizeof(z64);
        const cudaMemcpyKind kind = dp ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (want.sigL) CK(cudaMemcpyAsync(want.sigL + off_ss[w.idx], w.sig[0], cnt, kind, st), "copy sigma");
        if (want.sigR) CK(cudaMemcpyAsync(want.sigR + off_ss[w.idx], w.sig[1], cnt, kind, st), "copy sigma");
      }
    }

    // 2.-4. sweeps, boundary, transmission (or the density of states)
    std::vector<int> h_sinfo, h_binfo;
    std::vector<z64> h_tr(P);
    std::vector<double> ir_err(P, -1.0);
    if (want.dos) {
      h->plan_error = false;
      build_dos_sweeps(h, pts, sinfo, nmax);
      build_dos_diag(h, pts, binfo, h->dtr, nmax);
      if (h->plan_error) return fail(h, SS_ERR_OOM, "tensor-core packing buffer too small for the sweeps");
      CK(h->p_sweep.upload(st), "upload sweeps");
      CK(h->p_bound.upload(st), "upload diagonal blocks");
      CK(h->p_sweep.execute(st, &h->nlaunch, h->P(), h->cfg.use_graphs), "sweeps");
      CK(h->p_bound.execute(st, &h->nlaunch, h->P(), h->cfg.use_graphs), "diagonal blocks");
      launch_scaled_imag(h->dtr, dosv, P * nmax, -1.0 / M_PI, st);
      ++h->nlaunch;
      CK(cudaGetLastError(), "density of states");
      for (int p = 0; p < P; ++p) {
        const PW& w = pts[p];
        CK(cudaMemcpyAsync(want.dos_out + off_n[w.idx], dosv + (size_t)p * nmax, sizeof(double) * w.n,
                           dp ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st), "copy dos");
      }
      h_sinfo.assign(2 * (size_t)P * nmax, 0);
      h_binfo.assign((size_t)P * nmax, 0);
      CK(cudaMemcpyAsync(h_sinfo.data(), sinfo, sizeof(int) * h_sinfo.size(), cudaMemcpyDeviceToHost, st), "info");
      CK(cudaMemcpyAsync(h_binfo.data(), binfo, sizeof(int) * h_binfo.size(), cudaMemcpyDeviceToHost, st), "info");
    }
    if (want.solve) {
      h->plan_error = false;
      build_sweeps(h, pts, sinfo, nsteps, refine);
      build_boundary(h, pts, want.x ? want.ninj : 0, binfo, h->dtr, refine);
      if (h->plan_error) return fail(h, SS_ERR_OOM, "tensor-core packing buffer too small for the sweeps");
      CK(h->p_sweep.upload(st), "upload sweeps");
      CK(h->p_bound.upload(st), "upload boundary");
      CK(h->p_sweep.execute(st, &h->nlaunch, h->P(), h->cfg.use_graphs), "sweeps");
      CK(h->p_bound.execute(st, &h->nlaunch, h->P(), h->cfg.use_graphs), "boundary");
      if (refine) {
        // FP64 iterative refinement of x until the normwise backward error
        // ||r|| / (||A - Sigma|| ||x|| + ||Inj||) (Frobenius norms) is <= ir_tol
        build_ir_residual(h, pts, want.ninj, rr, xx);
        build_ir_correction(h, pts, want.ninj, nsteps);
        if (h->plan_error) return fail(h, SS_ERR_OOM, "tensor-core packing buffer too small for the refinement");
        Plan nrm;
        build_ir_norms(nrm, pts, want.ninj, mm, bb);
        CK(nrm.upload(st), "upload");
        CK(nrm.run(st, &h->nlaunch, h->P()), "||A - Sigma||, ||Inj||");
        CK(h->p_ir_res.upload(st), "upload");
        CK(h->p_ir_cor.upload(st), "upload");
        std::vector<double> hr(P), hb(P), hm(P), hx(P);
        CK(cudaMemcpyAsync(hb.data(), bb, sizeof(double) * P, cudaMemcpyDeviceToHost, st), "read");
        CK(cudaMemcpyAsync(hm.data(), mm, sizeof(double) * P, cudaMemcpyDeviceToHost, st), "read");
        double prev = HUGE_VAL;
        for (int it = 0;; ++it) {
          CK(h->p_ir_res.execute(st, &h->nlaunch, h->P(), h->cfg.use_graphs), "residual");
          CK(cudaMemcpyAsync(hr.data(), rr, sizeof(double) * P, cudaMemcpyDeviceToHost, st), "read");
          CK(cudaMemcpyAsync(hx.data(), xx, sizeof(double) * P, cudaMemcpyDeviceToHost, st), "read");
          CK(cudaStreamSynchronize(st), "refinement sync");
          double worst_rel = 0.0;
          for (int p = 0; p < P; ++p) {
            const double den = std::sqrt(hm[p]) * std::sqrt(hx[p]) + std::sqrt(hb[p]);
            const double rel = std::sqrt(hr[p]) / std::max(den, 1e-300);
            ir_err[p] = rel;
            worst_rel = std::max(worst_rel, std::isfinite(rel) ? rel : 1e300);
          }
          // stop at the tolerance, at the cap, or when a correction no longer
          // halves the residual (FP64 working accuracy: more steps cannot help)
          if (worst_rel <= h->cfg.ir_tol || it >= h->cfg.ir_max_iter || worst_rel > 0.5 * prev) break;
          prev = worst_rel;
          CK(h->p_ir_cor.execute(st, &h->nlaunch, h->P(), h->cfg.use_graphs), "correction");
        }
      }
      h_sinfo.assign(n_sinfo, 0);
      h_binfo.assign(P, 0);
      CK(cudaMemcpyAsync(h_sinfo.data(), sinfo, sizeof(int) * h_sinfo.size(), cudaMemcpyDeviceToHost, st), "info");
      CK(cudaMemcpyAsync(h_binfo.data(), binfo, sizeof(int) * P, cudaMemcpyDeviceToHost, st), "info");
      CK(cudaMemcpyAsync(h_tr.data(), h->dtr, sizeof(z64) * P, cudaMemcpyDeviceToHost, st), "read T");
      if (want.x && !dp) {
        for (auto& w : pts) {
          const size_t cnt = (size_t)w.n * w.s * want.ninj * sizeof(z64);
          CK(cudaMemcpyAsync(want.x + off_x[w.idx], w.x, cnt, cudaMemcpyDeviceToHost, st), "copy x");
        }
      }
    }
    CK(cudaStreamSynchronize(st), "pipeline sync");
    CK(cudaGetLastError(), "pipeline");
    if (h->cfg.profile) h->prof.collect();

    for (int p = 0; p < P; ++p) {
      const PW& w = pts[p];
      const int i = w.idx;
      iters[2 * i] = h_it[2 * p];
      iters[2 * i + 1] = h_it[2 * p + 1];
      int stt = SS_OK;
      if (!reuse_sigma) {
        if (!h_conv[2 * p] || !h_conv[2 * p + 1]) stt = SS_ERR_NOT_CONVERGED;
        for (int q = 0; q < 4; ++q)
          if (h_dinfo[(q < 2 ? 2 * p + q : 2 * P + 2 * p + q - 2)] && stt == SS_OK) stt = SS_ERR_SINGULAR;
      }
      if (want.dos) {
        bool bad = false;
        for (int d = 0; d < 2; ++d)
          for (int t = 0; t < nmax; ++t) bad = bad || h_sinfo[(size_t)(2 * p + d) * nmax + t] != 0;
        for (int t = 0; t < w.n; ++t) bad = bad || h_binfo[(size_t)p * nmax + t] != 0;
        if (bad && stt == SS_OK) {
          stt = SS_ERR_SINGULAR;
          if (h->err.empty()) h->err = "singular block in the density of states of point " + std::to_string(i);
        }
      }
      if (want.solve) {
        for (int j = 0; j < w.np && stt == SS_OK; ++j)
          for (int d = 0; d < 2 && stt == SS_OK; ++d)
            for (int t = 0; t < nsteps; ++t)
              if (h_sinfo[sinfo_index(p, j, d, t, nsteps)]) {
                stt = SS_ERR_SINGULAR;
                if (h->err.empty())
                  h->err = "singular diagonal block in the sweep of point " + std::to_string(i);
                break;
              }
        if (h_binfo[p] && stt == SS_OK) stt = SS_ERR_SINGULAR;
        if (ir_err[p] >= 0.0) {
          err_out[i] = ir_err[p];
          if (stt == SS_OK && !(ir_err[p] <= h->cfg.ir_tol)) stt = SS_ERR_NOT_CONVERGED;
        }
        if (stt == SS_OK && !(std::isfinite(h_tr[p].x) && std::isfinite(h_tr[p].y))) {
          stt = SS_ERR_SINGULAR;
          h->err = "non-finite transmission at point " + std::to_string(i);
        }
        T[i] = h_tr[p].x;
        Ti[i] = h_tr[p].y;
      }
      status[i] = stt;
      rc_all = worst(rc_all, stt);
    }
  }
  // cache
  h->cE.assign(E, E + n_pts);
  h->cK.assign(k_id, k_id + n_pts);
  h->c_sigma = one_batch;
  h->c_iters = iters;
  h->c_T = want.solve && n_pts <= h->cfg.max_points;
  h->cT = T;
  h->cTi = Ti;
  h->c_status = status;
  h->c_err = err_out;
  return rc_all;
}

}  // namespace

namespace ss {
size_t caroli_scratch_elems(int n_pts, int s) { return (size_t)n_pts * (4 * (size_t)s * s + 1); }

void caroli_descriptors(int n_pts, int s, const z64* sigL, const z64* sigR, const z64* G, z64* scratch,
                        std::vector<FormDesc>& f, std::vector<GemmDesc>& g, std::vector<TraceDesc>& t) {
  const size_t ss2 = (size_t)s * s;
  z64* traces = scratch + (size_t)n_pts * 4 * ss2;
  for (int p = 0; p < n_pts; ++p) {
    z64* base = scratch + (size_t)p * 4 * ss2;
    z64 *gl = base, *gr = base + ss2, *m1 = base + 2 * ss2, *m2 = base + 3 * ss2;
    const z64* sig[2] = {sigL + p * ss2, sigR + p * ss2};
    z64* gam[2] = {gl, gr};
    for (int q = 0; q < 2; ++q) {
      FormDesc gm = fdesc(gam[q], s, s, s);
      gm.x = sig[q]; gm.ldx = s; gm.ax = make_double2(0.0, 1.0);
      gm.y = sig[q]; gm.ldy = s; gm.ty = 1; gm.ay = make_double2(0.0, -1.0);
      f.push_back(gm);
    }
    const z64* Gp = G + p * ss2;
    g.push_back(gdesc(s, s, s, plain(gl, s), plain(Gp, s), m1, s, ONE, ZERO));
    g.push_back(gdesc(s, s, s, plain(gr, s), plain(Gp, s, 1), m2, s, ONE, ZERO));
    t.push_back({m1, s, m2, s, s, traces + p, nullptr});
  }
}
}  // namespace ss

// ======================================================================= C ABI
extern "C" {

void ss_config_default(ss_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->n_b_max = 64;
  cfg->s_b_max = 512;
  cfg->max_points = 8;
  cfg->max_inj = 64;
  cfg->precision = SS_FP64;
  cfg->eta = 1e-10;
  cfg->decim_tol = 1e-14;
  cfg->decim_max_iter = 100;
  cfg->ir_tol = 1e-14;
  cfg->ir_max_iter = 10;
  cfg->warm_start = 0;
  cfg->stream = nullptr;
  cfg->device_ptrs = 0;
  cfg->use_graphs = 1;
  cfg->profile = 0;
  cfg->partitions = 1;
  cfg->memory_lean = 0;
  cfg->hermitian_sweeps = 0;
  cfg->obc = SS_OBC_DECIMATION;
  cfg->feast_radius = 50.0;
  cfg->feast_points = 16;
  cfg->feast_subspace = 0;
  cfg->tournament_pivoting = 0;
  cfg->lu_lookahead = 0;
}

int ss_create(ss_handle** hp, const ss_config* cfg) {
  if (!hp) { g_create_error = "NULL handle pointer"; return SS_ERR_ARG; }
  *hp = nullptr;
  if (!cfg) { g_create_error = "NULL config"; return SS_ERR_ARG; }
  if (cfg->n_b_max < 1 || cfg->s_b_max < 1 || cfg->max_points < 1 || cfg->max_inj < 0) {
    g_create_error = "non-positive workspace sizes";
    return SS_ERR_ARG;
  }
  if (cfg->precision != SS_FP64 && cfg->precision != SS_MIXED_OZAKI) {
    // The 3/6-product split modes (about 5e-6 relative) are available through
    // ss_zgemm only: the lead doubling at eta = 1e-10 amplifies their error to
    // O(1) in band, so the pipeline takes FP64-accurate products.
    g_create_error = "pipeline precision must be SS_FP64 or SS_MIXED_OZAKI";
    return SS_ERR_ARG;
  }
  if (!(cfg->eta >= 0.0) || !(cfg->decim_tol >= 0.0) || cfg->decim_max_iter < 1) {
    g_create_error = "invalid eta / decim_tol / decim_max_iter";
    return SS_ERR_ARG;
  }
  if (cfg->obc != SS_OBC_DECIMATION && cfg->obc != SS_OBC_FEAST) {
    g_create_error = "obc must be SS_OBC_DECIMATION or SS_OBC_FEAST";
    return SS_ERR_ARG;
  }
  if (cfg->obc == SS_OBC_FEAST &&
      (!(cfg->feast_radius > 1.0) || cfg->feast_points < 2 || cfg->feast_subspace < 0 ||
       2 * cfg->s_b_max > 512 + (cfg->feast_subspace > 0 ? 1 << 30 : 0) || cfg->feast_subspace > 512)) {
    g_create_error = "contour solver: radius > 1, points >= 2, subspace 0..512 (0: 2 s_b, needs s_b <= 256)";
    return SS_ERR_ARG;
  }
  if (cfg->partitions < 1 || cfg->partitions > MAXP) {
    g_create_error = "partitions outside 1.." + std::to_string(MAXP);
    return SS_ERR_ARG;
  }
  if (cfg->lu_lookahead != 0 && cfg->lu_lookahead != 1) {
    g_create_error = "lu_lookahead must be 0 or 1";
    return SS_ERR_ARG;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev < 1) {
    g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return SS_ERR_CUDA;
  }
  std::unique_ptr<ss_handle> h(new ss_handle());
  h->cfg = *cfg;
  cudaGetDevice(&h->device);
  if (cfg->stream) {
    h->stream = (cudaStream_t)cfg->stream;
  } else {
    e = cudaStreamCreate(&h->stream);
    if (e != cudaSuccess) { g_create_error = cudaGetErrorString(e); return SS_ERR_CUDA; }
    h->own_stream = true;
  }
  h->arena_bytes = (size_t)cfg->max_points *
                   point_bytes(cfg->n_b_max, cfg->s_b_max, cfg->max_inj, cfg->precision == SS_MIXED_OZAKI,
                               cfg->memory_lean ? LAYOUT_LEAN : LAYOUT_FULL, cfg->partitions);
  e = cudaMalloc(&h->arena, h->arena_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (h->own_stream) cudaStreamDestroy(h->stream);
    g_create_error = "workspace of " + std::to_string(h->arena_bytes) + " bytes: " + cudaGetErrorString(e);
    return SS_ERR_OOM;
  }
  if (h->mixed()) {
    // the largest tensor-core group: the doubling products, 4 GEMMs per lead
    // with 2 distinct A (s rows) and 2 distinct B (2s rows) operands, each
    // sliced into S slices of width w
    const int s = cfg->s_b_max;
    OzShape sh;
    oz_plan(s, &sh);
    const size_t a1 = (((size_t)s * sh.S * sh.w * 2) + 1023) & ~size_t(1023);
    const size_t b1 = (((size_t)2 * s * sh.S * sh.w * 2) + 1023) & ~size_t(1023);
    const size_t ex = (((size_t)s * sizeof(int)) + 1023) & ~size_t(1023);
    const size_t per_lead = 2 * (a1 + ex) + 2 * (b1 + ex);
    h->pack_bytes = (size_t)cfg->max_points * 2 * per_lead + (4 << 20);
    // the partition merge's largest single product: R^-1 (2 np s square) times
    // the refinement's SMW right-hand side
    const int np = std::min(cfg->partitions, cfg->n_b_max);
    if (np > 1) {
      const int S2 = 2 * np * s;
      GemmDesc g{};
      g.m = S2; g.n = std::max(cfg->max_inj, 1); g.k = S2;
      static const z64 da = {0.0, 0.0}, db = {0.0, 0.0};
      g.a.p = &da; g.b.p = &db;
      h->pack_bytes = std::max(h->pack_bytes, Plan::oz_pack_bytes(std::vector<GemmDesc>(1, g)) + (4 << 20));
    }
    e = cudaMalloc(&h->pack, h->pack_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->tc_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->tc_err, 0, sizeof(int));
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(h->arena);
      cudaFree(h->pack);
      if (h->own_stream) cudaStreamDestroy(h->stream);
      g_create_error = "tensor-core packing buffer: " + std::string(cudaGetErrorString(e));
      return SS_ERR_OOM;
    }
  }
  *hp = h.release();
  return SS_OK;
}

int ss_set_hamiltonian(ss_handle* h, int k_id, int n_b, int s_b, const ss_c64* H_diag, const ss_c64* H_upper,
                       const ss_c64* S_diag, const ss_c64* S_upper, const ss_c64* lead_L, const ss_c64* lead_R) {
  if (!h) return SS_ERR_ARG;
  h->err.clear();
  if (k_id < 0 || k_id >= MAX_K_ID) return fail(h, SS_ERR_ARG, "k_id outside 0..4095");
  if (n_b < 1 || s_b < 1 || n_b > h->cfg.n_b_max || s_b > h->cfg.s_b_max)
    return fail(h, SS_ERR_ARG, "n_b / s_b outside 1..(n_b_max, s_b_max)");
  if (!H_diag || !S_diag || (n_b > 1 && (!H_upper || !S_upper)))
    return fail(h, SS_ERR_ARG, "NULL Hamiltonian block array");
  if (n_b < 2 && (!lead_L || !lead_R)) return fail(h, SS_ERR_ARG, "periodic leads need n_b >= 2");
  auto it = h->ks.find(k_id);
  if (it != h->ks.end()) { it->second.free_all(); h->ks.erase(it); }
  h->c_sigma = h->c_T = false;
  h->cE.clear();
  KData kd;
  kd.n = n_b; kd.s = s_b;
  const size_t ss2 = (size_t)s_b * s_b;
  const cudaMemcpyKind kind = h->cfg.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaStream_t st = h->stream;
  auto alloc_copy = [&](z64** dst, const ss_c64* src, size_t cnt) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(cnt, 1) * sizeof(z64));
    if (e != cudaSuccess || cnt == 0) return e;
    return cudaMemcpyAsync(*dst, src, cnt * sizeof(z64), kind, st);
  };
  cudaError_t e = alloc_copy(&kd.Hd, H_diag, n_b * ss2);
  if (e == cudaSuccess) e = alloc_copy(&kd.Sd, S_diag, n_b * ss2);
  if (e == cudaSuccess) e = alloc_copy(&kd.Hu, H_upper, (n_b - 1) * ss2);
  if (e == cudaSuccess) e = alloc_copy(&kd.Su, S_upper, (n_b - 1) * ss2);
  if (e == cudaSuccess && (lead_L || lead_R)) e = cudaMalloc(&kd.lead, 8 * ss2 * sizeof(z64));
  if (e == cudaSuccess && lead_L) e = cudaMemcpyAsync(kd.lead, lead_L, 4 * ss2 * sizeof(z64), kind, st);
  if (e == cudaSuccess && lead_R) e = cudaMemcpyAsync(kd.lead + 4 * ss2, lead_R, 4 * ss2 * sizeof(z64), kind, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    kd.free_all();
    if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return fail(h, SS_ERR_OOM, "Hamiltonian storage"); }
    return cuda_fail(h, e, "ss_set_hamiltonian");
  }
  for (int q = 0; q < 2; ++q) {
    const ss_c64* given = q == 0 ? lead_L : lead_R;
    if (given) {
      z64* base = kd.lead + (size_t)q * 4 * ss2;
      for (int j = 0; j < 4; ++j) kd.cell[q][j] = base + j * ss2;
    } else {
      const int cellb = q == 0 ? 0 : n_b - 1;       // end cell
      const int upb = q == 0 ? 0 : n_b - 2;         // its coupling block
      kd.cell[q][0] = kd.Hd + cellb * ss2;
      kd.cell[q][1] = kd.Hu + upb * ss2;
      kd.cell[q][2] = kd.Sd + cellb * ss2;
      kd.cell[q][3] = kd.Su + upb * ss2;
    }
  }
  h->ks[k_id] = kd;
  return SS_OK;
}

// Counts the host-side launch calls of one public call into h->nhost.
struct HostCalls {
  ss_handle* h;
  long long c0;
  explicit HostCalls(ss_handle* hh) : h(hh), c0(host_launch_calls()) {}
  ~HostCalls() { if (h) h->nhost += host_launch_calls() - c0; }
};

int ss_self_energy(ss_handle* h, int n_pts, const double* E, const int* k_id, ss_c64* sigma_L, ss_c64* sigma_R,
                   int* iters, int* status) {
  if (!h) return SS_ERR_ARG;
  HostCalls hc(h);
  h->err.clear();
  Want w;
  w.sigma_out = true;
  w.sigL = sigma_L;
  w.sigR = sigma_R;
  std::vector<int> st, it;
  std::vector<double> T, Ti;
  int rc = run_points(h, n_pts, E, k_id, w, st, it, T, Ti);
  if (rc == SS_ERR_ARG || rc == SS_ERR_STATE || rc == SS_ERR_CUDA || rc == SS_ERR_OOM) {
    if (st.empty()) return rc;
  }
  if (iters) for (size_t i = 0; i < it.size(); ++i) iters[i] = it[i];
  if (status) for (size_t i = 0; i < st.size(); ++i) status[i] = st[i];
  if (rc == SS_OK) h->c_T = false;
  return rc;
}

int ss_solve(ss_handle* h, int n_pts, const double* E, const int* k_id, int n_inj, const ss_c64* inj, ss_c64* x,
             int* status) {
  if (!h) return SS_ERR_ARG;
  HostCalls hc(h);
  h->err.clear();
  if (n_inj < 1 || n_inj > h->cfg.max_inj) return fail(h, SS_ERR_ARG, "n_inj outside 1..max_inj");
  if (!inj) return fail(h, SS_ERR_ARG, "NULL injection");
  Want w;
  w.solve = true;
  w.ninj = n_inj;
  w.inj = inj;
  w.x = x;
  std::vector<int> st, it;
  std::vector<double> T, Ti;
  int rc = run_points(h, n_pts, E, k_id, w, st, it, T, Ti);
  if (status) for (size_t i = 0; i < st.size(); ++i) status[i] = st[i];
  return rc;
}

int ss_transmission(ss_handle* h, int n_pts, const double* E, const int* k_id, double* T, double* err_est,
                    int* status) {
  if (!h) return SS_ERR_ARG;
  HostCalls hc(h);
  h->err.clear();
  if (!T && n_pts > 0) return fail(h, SS_ERR_ARG, "NULL T");
  std::vector<double> Tv, Ti;
  std::vector<int> st, it;
  int rc = SS_OK;
  if (h->c_T && same_points(h, n_pts, E, k_id)) {
    Tv = h->cT;
    Ti = h->cTi;
    st = h->c_status;
    for (int v : st) rc = worst(rc, v);
  } else {
    Want w;
    w.solve = true;
    rc = run_points(h, n_pts, E, k_id, w, st, it, Tv, Ti);
    if (st.empty()) return rc;
  }
  std::vector<double> err(n_pts);
  for (int i = 0; i < n_pts; ++i) {
    err[i] = std::fabs(Ti[i]) / std::max(1.0, std::fabs(Tv[i]));
    if (h->mixed() && (int)h->c_err.size() == n_pts && h->c_err[i] >= 0.0) err[i] = std::max(err[i], h->c_err[i]);
  }
  if (h->cfg.device_ptrs) {
    cudaError_t e = cudaMemcpyAsync(T, Tv.data(), sizeof(double) * n_pts, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && err_est)
      e = cudaMemcpyAsync(err_est, err.data(), sizeof(double) * n_pts, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy T");
  } else {
    std::memcpy(T, Tv.data(), sizeof(double) * n_pts);
    if (err_est) std::memcpy(err_est, err.data(), sizeof(double) * n_pts);
  }
  if (status) for (int i = 0; i < n_pts; ++i) status[i] = st[i];
  return rc;
}

int ss_dos(ss_handle* h, int n_pts, const double* E, const int* k_id, double* dos, int* status) {
  if (!h) return SS_ERR_ARG;
  HostCalls hc(h);
  h->err.clear();
  if (!dos && n_pts > 0) return fail(h, SS_ERR_ARG, "NULL dos");
  Want w;
  w.dos = true;
  w.dos_out = dos;
  std::vector<int> st, it;
  std::vector<double> T, Ti;
  int rc = run_points(h, n_pts, E, k_id, w, st, it, T, Ti);
  if (status) for (size_t i = 0; i < st.size(); ++i) status[i] = st[i];
  h->c_T = false;
  return rc;
}

int ss_autotune(ss_handle* h, int s_b, int n_problems, const char* cache_path, int* nb_out, int* nbo_out,
                int* upd_out, double* ms_out) {
  if (!h) return SS_ERR_ARG;
  h->err.clear();
  if (s_b < 1 || s_b > h->cfg.s_b_max || n_problems < 1) return fail(h, SS_ERR_ARG, "ss_autotune: bad sizes");
  const int prec = h->cfg.precision;
  auto report = [&](const ss_handle::Tune& t) {
    if (nb_out) *nb_out = t.nb;
    if (nbo_out) *nbo_out = t.nbo;
    if (upd_out) *upd_out = t.upd;
    if (ms_out) *ms_out = t.ms;
    return SS_OK;
  };
  // cache lines: "<precision> <s_b> <n_problems> <nb> <nbo> <upd> <ms>" (LU blocking)
  // and "G <precision> <s_b> <n_problems> <square tile> <update tile>" (FP64 GEMM tiles)
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      int pr, sb, np, nb, nbo, upd, gs, gu;
      double ms;
      bool hit = false, ghit = false;
      ss_handle::Tune t{};
      int tgs = -1, tgu = -1;
      char line[256];
      while (std::fgets(line, sizeof line, f)) {
        if (std::sscanf(line, "G %d %d %d %d %d", &pr, &sb, &np, &gs, &gu) == 5) {
          if (pr == prec && sb == s_b && np == n_problems) { tgs = gs; tgu = gu; ghit = true; }
        } else if (std::sscanf(line, "%d %d %d %d %d %d %lf", &pr, &sb, &np, &nb, &nbo, &upd, &ms) == 7) {
          if (pr == prec && sb == s_b && np == n_problems) { t = {nb, nbo, upd, ms}; hit = true; }
        }
      }
      std::fclose(f);
      if (hit) {  // a cache without tile lines keeps the heuristic tile shapes
        t.gsq = ghit ? tgs : -1;
        t.gup = ghit ? tgu : -1;
        h->tune[s_b] = t;
        return report(t);
      }
    }
  }
  // synthetic batch of [D | B] systems, D diagonally weighted so the
  // factorisation is well posed; a pristine copy restores it between runs
  const size_t per = (size_t)s_b * 3 * s_b;  // [D | B], B of 2 s_b columns like the doubling and sweeps
  const size_t tot = per * n_problems;
  z64 *W = nullptr, *W0 = nullptr;
  int *piv = nullptr, *info = nullptr;
  cudaStream_t st = h->stream;
  CK(cudaMalloc(&W, tot * sizeof(z64)), "autotune buffer");
  cudaError_t e = cudaMalloc(&W0, tot * sizeof(z64));
  if (e == cudaSuccess) e = cudaMalloc(&piv, (size_t)n_problems * s_b * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&info, (size_t)n_problems * sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(W); cudaFree(W0); cudaFree(piv); cudaFree(info);
    return cuda_fail(h, e, "autotune buffer");
  }
  {
    std::vector<z64> host(tot);
    unsigned long long r = 12345;
    for (size_t i = 0; i < tot; ++i) {
      r = r * 6364136223846793005ull + 1442695040888963407ull;
      const double a = ((double)((r >> 11) & ((1ull << 52) - 1)) / (double)(1ull << 52)) - 0.5;
      r = r * 6364136223846793005ull + 1442695040888963407ull;
      const double b = ((double)((r >> 11) & ((1ull << 52) - 1)) / (double)(1ull << 52)) - 0.5;
      host[i] = make_double2(a, b);
    }
    for (int p = 0; p < n_problems; ++p)
      for (int i = 0; i < s_b; ++i) host[p * per + (size_t)i * 3 * s_b + i].x += 4.0;
    e = cudaMemcpy(W0, host.data(), tot * sizeof(z64), cudaMemcpyHostToDevice);
  }
  std::vector<ss_handle::Tune> cands;
  const int nbs[2] = {8, s_b <= 512 ? 16 : 32};
  for (int nb : nbs) {
    cands.push_back({nb, 0, (int)Plan::UPD_FP64, 0.0});
    if (h->mixed()) {
      cands.push_back({nb, 0, (int)Plan::UPD_EXACT_TC, 0.0});
      for (int nbo : {32, 64, 128, 256})
        if (nbo < s_b && nbo > nb)
          for (int u : {(int)Plan::UPD_EXACT_TC, (int)Plan::UPD_EXACT_FAR, (int)Plan::UPD_EXACT_ALL})
            cands.push_back({nb, nbo, u, 0.0});
    }
  }
  ss_handle::Tune best{-1, 0, 0, 0.0};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // one LU solve of the batch with blocking c and update tile shape var_up
  // (-1: the heuristic), timed as the pipeline runs it (replayed from a CUDA
  // graph captured on the first run); best of three after a warm-up run
  auto time_lu = [&](const ss_handle::Tune& c, int var_up) {
    std::vector<LuDesc> ds;
    for (int p = 0; p < n_problems; ++p) {
      LuDesc L{};
      L.w = W + p * per; L.ldw = 3 * s_b; L.s = s_b; L.ncols = 3 * s_b; L.ipiv = piv + (size_t)p * s_b; L.info = info + p;
      ds.push_back(L);
    }
    Plan P;
    P.set_gemm_variants(-1, var_up);
    if (!P.lu_solve(ds, c.nb, (Plan::Updates)c.upd, h->pack, h->pack_bytes, h->tc_err, c.nbo, 0,
                    h->cfg.lu_lookahead))
      return -1.f;
    e = P.upload(st);
    float best_ms = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      e = cudaMemcpyAsync(W, W0, tot * sizeof(z64), cudaMemcpyDeviceToDevice, st);
      cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = h->cfg.use_graphs ? P.replay(st, nullptr) : P.run(st, nullptr);
      cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best_ms = std::min(best_ms, ms);  // first run warms up
    }
    return best_ms;
  };
  for (auto& c : cands) {
    if (e != cudaSuccess) break;
    const float ms = time_lu(c, -1);
    if (ms < 0.f) continue;
    c.ms = ms;
    if (e == cudaSuccess && (best.nb < 0 || c.ms < best.ms)) best = c;
  }
  // FP64 GEMM tile shapes.  The products of full s x s blocks (FP64 path):
  // one group of n_problems products timed with the heuristic (-1) and with
  // every tile shape.  The LU's wide rank-nb updates: the whole LU solve of
  // the chosen blocking timed with each shape for them (they come in several
  // shapes: the outer block's rows right of it, the back substitution's rows
  // above it).  The fastest replaces the padded-work heuristic.
  auto time_gemm = [&](const std::vector<GemmDesc>& g, bool lu_label) {
    int bv = -1;
    float bms = 1e30f;
    for (int v = -1; v < zgemm_num_variants() && e == cudaSuccess; ++v) {
      Plan G;
      G.gemm(g, lu_label, v);
      e = G.upload(st);
      float vbest = 1e30f;
      for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        e = G.run(st, nullptr);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) vbest = std::min(vbest, ms);
      }
      if (e == cudaSuccess && vbest < bms) { bms = vbest; bv = v; }
    }
    return bv;
  };
  if (e == cudaSuccess && best.nb > 0) {
    if (prec == SS_FP64) {
      std::vector<GemmDesc> gsq;
      for (int p = 0; p < n_problems; ++p) {
        z64* Wp = W + p * per;
        gsq.push_back(gdesc(s_b, s_b, s_b, plain(Wp, 3 * s_b), plain(Wp + s_b, 3 * s_b), Wp + 2 * s_b, 3 * s_b, ONE, ZERO));
      }
      best.gsq = time_gemm(gsq, false);
    }
    float bms = best.ms;  // the heuristic's time from the blocking search
    best.gup = -1;
    for (int v = 0; v < zgemm_num_variants() && e == cudaSuccess; ++v) {
      const float ms = time_lu(best, v);
      if (e == cudaSuccess && ms >= 0.f && ms < bms) { bms = ms; best.gup = v; }
    }
    best.ms = bms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(W); cudaFree(W0); cudaFree(piv); cudaFree(info);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune run");
  if (best.nb < 0) return fail(h, SS_ERR_OOM, "no candidate fits the packing buffer");
  h->tune[s_b] = best;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "%d %d %d %d %d %d %.6f\n", prec, s_b, n_problems, best.nb, best.nbo, best.upd, best.ms);
      std::fprintf(f, "G %d %d %d %d %d\n", prec, s_b, n_problems, best.gsq, best.gup);
      std::fclose(f);
    }
  }
  return report(best);
}

int ss_set_momentum(ss_handle* h, int k_id, double k) {
  if (!h) return SS_ERR_ARG;
  h->err.clear();
  auto it = h->ks.find(k_id);
  if (it == h->ks.end()) return fail(h, SS_ERR_STATE, "no Hamiltonian set for k_id " + std::to_string(k_id));
  if (!std::isfinite(k)) return fail(h, SS_ERR_ARG, "non-finite momentum");
  it->second.kval = k;
  h->c_sigma = h->c_T = false;
  return SS_OK;
}

int ss_set_warm_start(ss_handle* h, ss_mlp* net, int side, double out_scale) {
  if (!h) return SS_ERR_ARG;
  if (side < 0 || side > 1 || !(out_scale > 0.0)) return fail(h, SS_ERR_ARG, "side must be 0/1, out_scale > 0");
  h->warm_net[side] = net;
  h->warm_scale[side] = out_scale;
  h->c_sigma = h->c_T = false;
  return SS_OK;
}

int ss_surface_gf(ss_handle* h, int n_pts, const double* E, const int* k_id, const double* kval, int side,
                  int use_warm, int warm_iters, double warm_tol, ss_c64* g, int* iters, int* seeded, int* status) {
  if (!h) return SS_ERR_ARG;
  h->err.clear();
  if (n_pts < 0 || side < 0 || side > 1 || !E || !k_id || !g || warm_iters < 0)
    return fail(h, SS_ERR_ARG, "ss_surface_gf: bad arguments");
  if (n_pts == 0) return SS_OK;
  ss_mlp* net = use_warm ? h->warm_net[side] : nullptr;
  if (use_warm && !net) return fail(h, SS_ERR_STATE, "no warm-start network attached for this side");
  if (net && !kval) return fail(h, SS_ERR_ARG, "kval is required with the warm start");
  int n_in = 0, n_out = 0, mb = 0;
  if (net) mlp_dims(net, &n_in, &n_out, &mb);
  const bool dp = h->cfg.device_ptrs != 0;
  cudaStream_t st = h->stream;
  const int P_max = h->cfg.max_points;
  int rc_all = SS_OK;
  size_t gofs = 0;
  for (int base = 0; base < n_pts; base += P_max) {
    const int P = std::min(P_max, n_pts - base);
    std::vector<PW> pts(P);
    Carve c(h->arena);
    int smax = 0;
    for (int p = 0; p < P; ++p) {
      auto it = h->ks.find(k_id[base + p]);
      if (it == h->ks.end()) return fail(h, SS_ERR_STATE, "no Hamiltonian for k_id " + std::to_string(k_id[base + p]));
      PW& w = pts[p];
      w.idx = base + p; w.n = it->second.n; w.s = it->second.s; w.E = E[base + p]; w.kd = &it->second;
      carve_doubling(c, w);  // only the doubling buffers are used
      smax = std::max(smax, w.s);
    }
    if (c.off > h->arena_bytes) return fail(h, SS_ERR_OOM, "workspace too small for the chunk");
    const int NP = 2 * P;
    int rc = ensure_scalars(h, 2 * P * 3 + 4 * P, 3 * 2 * P, P);
    if (rc) return rc;
    int* act = h->dint;
    int* itr = act + NP;
    int* conv = itr + NP;
    int* dinfo = conv + NP;
    double* na = h->ddbl;
    double* nb = na + NP;
    double* nd = nb + NP;
    std::vector<int> accepted(P, 0);
    // ---------------- warm start: network seed, fixed-point steps, residual judge
    if (net) {
      std::vector<double> kv(P);
      for (int p = 0; p < P; ++p) kv[p] = kval[base + p];
      h->plan_error = false;
      rc = warm_seed(h, pts, side, kv, warm_iters, warm_tol, dinfo, accepted);
      if (rc) return rc;
    }
    // ---------------- plain doubling for the others (this lead only)
    std::vector<int> h_it(NP, 0), h_conv(NP, 1), h_dinfo(4 * P, 0), init(NP, 0);
    bool any = false;
    for (int p = 0; p < P; ++p)
      if (!accepted[p]) { init[2 * p + side] = 1; any = true; }
    if (any) {
      h->plan_error = false;
      // the accepted seeds keep their g in es[side]; the other lead is not needed
      std::vector<int> skip(NP, 0);
      for (int p = 0; p < P; ++p) { skip[2 * p + side] = accepted[p]; skip[2 * p + 1 - side] = 1; }
      build_decimation(h, pts, act, itr, conv, dinfo, na, nb, nd, true, &skip);
      // g = es^-1 for the lead: [es | 1] -> LU
      Plan& F = h->p_final_g;
      F.clear();
      std::vector<FormDesc> ff, fo;
      std::vector<LuDesc> lus;
      for (int p = 0; p < P; ++p) {
        if (accepted[p]) continue;
        PW& w = pts[p];
        const int s = w.s;
        z64* W = w.Wd[side];
        ff.push_back(fcopy(W, 2 * s, w.es[side], s, s, s));
        ff.push_back(fident(W + s, 2 * s, s, s, 1.0));
        LuDesc L{};
        L.w = W; L.ldw = 2 * s; L.s = s; L.ncols = 2 * s; L.ipiv = w.ipd[side]; L.info = dinfo + 2 * P + 2 * p + side;
        lus.push_back(L);
        fo.push_back(fcopy(w.T1[side], s, W + s, 2 * s, s, s));
      }
      F.form(ff);
      ::lu(h, F, lus);
      F.form(fo);
      if (h->plan_error) return fail(h, SS_ERR_OOM, "tensor-core packing buffer too small");
      CK(cudaMemcpyAsync(act, init.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, st), "flags");
      CK(h->p_setup.upload(st), "upload");
      CK(h->p_iter[0].upload(st), "upload");
      CK(h->p_iter[1].upload(st), "upload");
      CK(F.upload(st), "upload");
      CK(h->p_setup.run(st, &h->nlaunch, h->P()), "setup");
      std::vector<int> h_act(NP);
      for (int it = 0; it < h->cfg.decim_max_iter + 2; it += 2) {
        CK(h->p_iter[0].run(st, &h->nlaunch, h->P()), "doubling step");
        CK(h->p_iter[1].run(st, &h->nlaunch, h->P()), "doubling step");
        CK(cudaMemcpyAsync(h_act.data(), act, sizeof(int) * NP, cudaMemcpyDeviceToHost, st), "flags");
        CK(cudaStreamSynchronize(st), "sync");
        bool a2 = false;
        for (int v : h_act) a2 = a2 || v;
        if (!a2) break;
      }
      CK(F.run(st, &h->nlaunch, h->P()), "final g");
      CK(cudaMemcpyAsync(h_it.data(), itr, sizeof(int) * NP, cudaMemcpyDeviceToHost, st), "iters");
      CK(cudaMemcpyAsync(h_conv.data(), conv, sizeof(int) * NP, cudaMemcpyDeviceToHost, st), "conv");
    }
    CK(cudaMemcpyAsync(h_dinfo.data(), dinfo, sizeof(int) * 4 * P, cudaMemcpyDeviceToHost, st), "info");
    // outputs
    for (int p = 0; p < P; ++p) {
      PW& w = pts[p];
      const size_t cnt = (size_t)w.s * w.s;
      const z64* src = accepted[p] ? w.es[side] : w.T1[side];
      CK(cudaMemcpyAsync(g + gofs, src, cnt * sizeof(z64), dp ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st),
         "copy g");
      gofs += cnt;
    }
    CK(cudaStreamSynchronize(st), "surface gf sync");
    if (h->cfg.profile) h->prof.collect();
    for (int p = 0; p < P; ++p) {
      int stt = SS_OK;
      if (!accepted[p]) {
        if (!h_conv[2 * p + side]) stt = SS_ERR_NOT_CONVERGED;
        if (h_dinfo[2 * p + side] || h_dinfo[2 * P + 2 * p + side]) stt = SS_ERR_SINGULAR;
      }
      if (iters) iters[base + p] = accepted[p] ? warm_iters : h_it[2 * p + side];
      if (seeded) seeded[base + p] = accepted[p];
      if (status) status[base + p] = stt;
      rc_all = worst(rc_all, stt);
    }
  }
  h->c_sigma = h->c_T = false;
  return rc_all;
}

int ss_destroy(ss_handle* h) {
  if (!h) return SS_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& kv : h->ks) kv.second.free_all();
  h->ks.clear();
  cudaFree(h->arena);
  cudaFree(h->pack);
  cudaFree(h->tc_err);
  cudaFree(h->dint);
  cudaFree(h->ddbl);
  cudaFree(h->dtr);
  cudaFree(h->feat);
  cudaFree(h->warm_y);
  cudaFree(h->wres);
  cudaFree(h->feast_buf);
  cudaFree(h->feast_info);
  h->p_fa.clear(); h->p_fb.clear(); h->p_fc.clear();
  h->p_warm_iter.clear(); h->p_warm_judge.clear(); h->p_final_g.clear();
  h->p_ir_res.clear(); h->p_ir_cor.clear();
  h->p_setup.clear(); h->p_iter[0].clear(); h->p_iter[1].clear();
  h->p_final.clear(); h->p_sweep.clear(); h->p_bound.clear();
  h->prof.reset();
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return SS_OK;
}

const char* ss_last_error(const ss_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

long long ss_launch_count(const ss_handle* h) { return h ? h->nlaunch : 0; }

long long ss_host_launch_count(const ss_handle* h) { return h ? h->nhost : 0; }

int ss_exact_gemm_plan(int k, int* w, int* beta, int* S, int* npass, unsigned char* pd, unsigned char* pt0,
                       unsigned char* pnp) {
  if (k < 1) return SS_ERR_ARG;
  OzShape sh;
  oz_plan(k, &sh);
  if (sh.npass > OZ_MAXPASS) return SS_ERR_ARG;
  if (w) *w = sh.w;
  if (beta) *beta = sh.beta;
  if (S) *S = sh.S;
  if (npass) *npass = sh.npass;
  for (int p = 0; p < sh.npass; ++p) {
    if (pd) pd[p] = sh.pd[p];
    if (pt0) pt0[p] = sh.pt0[p];
    if (pnp) pnp[p] = sh.pnp[p];
  }
  return SS_OK;
}

int ss_zgemm(int precision, int m, int n, int k, const ss_c64* A, int lda, int transA, const ss_c64* B, int ldb,
             int transB, ss_c64* C, int ldc, void* stream) {
  if (m < 0 || n < 0 || k < 1 || !A || !B || !C || lda < 1 || ldb < 1 || ldc < n ||
      (precision != SS_FP64 && precision != SS_MIXED_BF16X3 && precision != SS_MIXED_BF16X6 &&
       precision != SS_MIXED_OZAKI)) {
    g_create_error = "ss_zgemm: bad arguments";
    return SS_ERR_ARG;
  }
  if (m == 0 || n == 0) return SS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  GemmDesc g = gdesc(m, n, k, plain(reinterpret_cast<const z64*>(A), lda, transA ? 1 : 0),
                     plain(reinterpret_cast<const z64*>(B), ldb, transB ? 1 : 0), reinterpret_cast<z64*>(C), ldc,
                     ONE, ZERO);
  std::vector<GemmDesc> ds(1, g);
  Plan plan;
  unsigned char* pack = nullptr;
  int* err = nullptr;
  cudaError_t e = cudaSuccess;
  if (precision == SS_FP64) {
    plan.gemm(ds);
  } else if (precision == SS_MIXED_OZAKI) {
    const size_t cap = Plan::oz_pack_bytes(ds);
    e = cudaMallocAsync(&pack, cap, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&err, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e != cudaSuccess) { cudaGetLastError(); g_create_error = "ss_zgemm: scratch"; return SS_ERR_OOM; }
    if (!plan.oz_gemm(ds, pack, cap, err)) e = cudaErrorInvalidValue;
  } else {
    const size_t cap = Plan::tc_pack_bytes(ds, precision);
    e = cudaMallocAsync(&pack, cap, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&err, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e != cudaSuccess) { cudaGetLastError(); g_create_error = "ss_zgemm: scratch"; return SS_ERR_OOM; }
    if (!plan.tc_gemm(ds, precision, pack, cap, err)) e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) e = plan.upload(st);
  if (e == cudaSuccess) e = plan.run(st, nullptr);
  int herr = 0;
  if (err && e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (pack) cudaFreeAsync(pack, st);
  if (err) cudaFreeAsync(err, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { g_create_error = std::string("ss_zgemm: ") + cudaGetErrorString(e); return SS_ERR_CUDA; }
  if (herr) { g_create_error = "ss_zgemm: tensor-core pipeline wait timed out"; return SS_ERR_TIMEOUT; }
  return SS_OK;
}

int ss_caroli_transmission(int n_pts, int s_b, const ss_c64* sigma_L, const ss_c64* sigma_R, const ss_c64* G1n,
                           double* T, void* stream) {
  if (n_pts < 0 || s_b < 1) { g_create_error = "ss_caroli_transmission: bad sizes"; return SS_ERR_ARG; }
  if (n_pts == 0) return SS_OK;
  if (!sigma_L || !sigma_R || !G1n || !T) { g_create_error = "ss_caroli_transmission: NULL array"; return SS_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  z64* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, caroli_scratch_elems(n_pts, s_b) * sizeof(z64), st);
  if (e != cudaSuccess) { cudaGetLastError(); g_create_error = "ss_caroli_transmission: scratch"; return SS_ERR_OOM; }
  std::vector<FormDesc> f;
  std::vector<GemmDesc> g;
  std::vector<TraceDesc> t;
  caroli_descriptors(n_pts, s_b, reinterpret_cast<const z64*>(sigma_L), reinterpret_cast<const z64*>(sigma_R),
                     reinterpret_cast<const z64*>(G1n), scratch, f, g, t);
  Plan plan;
  plan.form(f);
  plan.gemm(g);
  plan.trace(t);
  e = plan.upload(st);
  if (e == cudaSuccess) e = plan.run(st, nullptr);
  if (e == cudaSuccess) {
    launch_real_part(scratch + (size_t)n_pts * 4 * s_b * s_b, T, n_pts, st);
    e = cudaGetLastError();
  }
  cudaFreeAsync(scratch, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { g_create_error = std::string("ss_caroli_transmission: ") + cudaGetErrorString(e); return SS_ERR_CUDA; }
  return SS_OK;
}

int ss_profile_read(ss_handle* h, int kind, double* total_ms, double* flops, long long* launches) {
  if (!h) return SS_ERR_ARG;
  if (kind < 0 || kind >= K_MEMSET) return fail(h, SS_ERR_ARG, "unknown kernel kind");
  h->prof.collect();
  if (total_ms) *total_ms = h->prof.ms[kind];
  if (flops) *flops = h->prof.flops[kind];
  if (launches) *launches = h->prof.launches[kind];
  return SS_OK;
}

int ss_profile_read_issued(ss_handle* h, int kind, double* issued_flops) {
  if (!h) return SS_ERR_ARG;
  if (kind < 0 || kind >= K_MEMSET) return fail(h, SS_ERR_ARG, "unknown kernel kind");
  h->prof.collect();
  if (issued_flops) *issued_flops = h->prof.issued[kind];
  return SS_OK;
}

int ss_profile_reset(ss_handle* h) {
  if (!h) return SS_ERR_ARG;
  h->prof.reset();
  return SS_OK;
}

}  // extern "C"
