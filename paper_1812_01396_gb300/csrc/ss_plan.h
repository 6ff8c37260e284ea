// Launch plans: a recorded list of grouped kernel launches whose descriptors
// live in one device buffer.  A plan is built on the host, uploaded with a
// single copy and then run eagerly or captured once into a CUDA graph and
// replayed (the doubling iterations of the self-energy step).
#pragma once
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "ss_internal.cuh"
#include "ss_tc.h"

namespace ss {

// Host-side launch calls made by this thread through plans: one per eager
// kernel launch or memset, one per graph launch.
long long host_launch_calls();

// Launch kinds; the numbering is also the `kind` argument of ss_profile_read.
enum LaunchKind { K_GEMM = 0, K_FORM, K_LU_PANEL, K_LU_ROW, K_LU_BACK, K_NORM1, K_TRACE, K_CHECK,
                  K_FILL, K_PACK_A, K_PACK_B, K_TCGEMM, K_GEMM32, K_OZSCALE, K_OZPACK, K_OZGEMM, K_FROB2,
                  K_GEMM_LU, K_OZGEMM_LU, K_LU_HPANEL, K_EIG, K_MEMSET,
                  // not launches: K_FORK makes the side stream wait for the main one, K_JOIN
                  // the main stream for the side one (records with `side` set run on it)
                  K_FORK, K_JOIN };

struct LaunchRec {
  LaunchKind kind;
  size_t off = 0, toff = 0;  // descriptor / tile-table offsets in the plan buffer
  int nprob = 0, tiles = 0;
  int k0 = 0, nb = 0, maxc = 0, nbo = 0;
  double tol = 0.0;
  int cap = 0, count = 0, ival = 0;
  void* p[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t bytes = 0;
  int side = 0;  // 1: issued on the plan's side stream (between a K_FORK and a K_JOIN)
};

// Optional per-launch timing: a CUDA event pair around every launch, with
// the algorithmic flops of GEMM launches counted only for problems whose
// `active` flag (mirrored on the host) is set.
struct Prof {
  struct Rec { int kind; cudaEvent_t a, b; double flops, issued; };
  std::vector<Rec> recs;
  const int* act_dev = nullptr;   // device flag array the descriptors point into
  const int* act_host = nullptr;  // host mirror of it at launch time
  int nact = 0;
  double ms[K_MEMSET + 1] = {0};
  double flops[K_MEMSET + 1] = {0};
  double issued[K_MEMSET + 1] = {0};  // flops the tensor pipe executes (digit pairs, padded K)
  long long launches[K_MEMSET + 1] = {0};
  // Fold finished records into the totals (call after a stream sync).
  void collect() {
    for (auto& r : recs) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.kind] += t;
      flops[r.kind] += r.flops;
      issued[r.kind] += r.issued;
      launches[r.kind] += 1;
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    recs.clear();
  }
  void reset() {
    collect();
    for (int i = 0; i <= K_MEMSET; ++i) { ms[i] = 0; flops[i] = 0; issued[i] = 0; launches[i] = 0; }
  }
};

class Plan {
 public:
  ~Plan() { release(); }
  // Forget the recorded launches.  A captured graph is kept: if the next
  // recording has the same launch sequence (same kinds, grid sizes, offsets
  // and pointer arguments) and fits the same device buffer, upload() keeps it
  // and replay() launches it again with the new descriptor contents.
  void clear() {
    host_.clear();
    recs_.clear();
  }
  size_t push(const void* data, size_t bytes, size_t align = 16) {
    size_t off = (host_.size() + align - 1) & ~(align - 1);
    host_.resize(off + bytes);
    if (bytes && data) std::memcpy(host_.data() + off, data, bytes);
    else if (bytes) std::memset(host_.data() + off, 0, bytes);
    return off;
  }
  template <class D>
  size_t push_vec(const std::vector<D>& v, size_t align = 16) { return push(v.data(), v.size() * sizeof(D), align); }

  // fp32 = true: the FP32-arithmetic kernel (low-rank updates of the mixed path)
  // lu_label: account the launch as an LU update (profiling only)
  // Tile shapes of the FP64 GEMM chosen by ss_autotune (-1: the heuristic):
  // sq for the products of full blocks, up for the LU's rank-nb updates.
  void set_gemm_variants(int sq, int up) { var_sq_ = sq; var_up_ = up; }
  void gemm(const std::vector<GemmDesc>& ds, bool lu_label = false, int force_variant = -1) {
    if (ds.empty()) return;
    // the tuned shape applies to the class it was timed on: square products of
    // full blocks, or rank-nb updates at least as wide as tall
    const GemmDesc& g0 = ds[0];
    const int tuned = lu_label ? ((g0.k <= 32 && g0.n >= g0.m) ? var_up_ : -1)
                               : ((g0.m == g0.n && g0.k >= 64) ? var_sq_ : -1);
    const int variant = force_variant >= 0 ? force_variant : (tuned >= 0 ? tuned : zgemm_variant(ds));
    std::vector<int> start(ds.size());
    int tot = 0;
    for (size_t i = 0; i < ds.size(); ++i) { start[i] = tot; tot += zgemm_tiles(ds[i].m, ds[i].n, variant); }
    if (tot == 0) return;
    LaunchRec r;
    r.ival = variant;
    r.kind = lu_label ? K_GEMM_LU : K_GEMM;
    r.off = push_vec(ds);
    r.toff = push_vec(start);
    r.nprob = (int)ds.size();
    r.tiles = tot;
    recs_.push_back(r);
  }
  void form(const std::vector<FormDesc>& ds) {
    if (ds.empty()) return;
    std::vector<int> start(ds.size());
    int tot = 0;
    for (size_t i = 0; i < ds.size(); ++i) { start[i] = tot; tot += zform_tiles(ds[i].rows, ds[i].cols); }
    if (tot == 0) return;
    LaunchRec r;
    r.kind = K_FORM;
    r.off = push_vec(ds);
    r.toff = push_vec(start);
    r.nprob = (int)ds.size();
    r.tiles = tot;
    recs_.push_back(r);
  }
  // Complex GEMMs on the tensor cores (split-BF16, mode 1: 3 products,
  // mode 2: 6 products).  Operands are packed into the device buffer `pack`
  // (cap bytes, reused by every tc_gemm group of the plan: launches are
  // stream-ordered); identical operands of the group are packed once.
  // Returns false if the packed operands do not fit or a tensor map fails.
  bool tc_gemm(const std::vector<GemmDesc>& ds, int mode, unsigned char* pack, size_t cap, int* err);
  static size_t tc_pack_bytes(const std::vector<GemmDesc>& ds, int mode);
  // FP64-accurate complex GEMMs on the tensor cores (digit-sliced BF16, exact
  // FP32 accumulation); operands sliced into `pack` as for tc_gemm.
  // Groups whose slices exceed `cap` are issued as consecutive chunks.
  bool oz_gemm(const std::vector<GemmDesc>& ds, unsigned char* pack, size_t cap, int* err, bool lu_label = false);
  static size_t oz_pack_bytes(const std::vector<GemmDesc>& ds);
  // Blocked LU + solve of every problem in ds (panel width nb <= 32; nb <= 0
  // picks the width from the largest block of the group).
  // Arithmetic of the rank-nb trailing and back-substitution updates
  // (panels, pivots and triangular blocks always stay FP64).
  // UPD_EXACT_ALL: the nb-deep updates inside an outer block too.
  // UPD_EXACT_FAR: like UPD_EXACT_TC, and the outer block's rows on the columns
  // right of it (nb deep, wide) also exact; the updates inside the block stay FP64.
  enum Updates { UPD_FP64 = 0, UPD_EXACT_TC = 2, UPD_EXACT_ALL = 3, UPD_EXACT_FAR = 4 };
  // UPD_EXACT_TC slices the update operands into `pack` (cap bytes).
  // nbo > nb (a multiple of nb): two-level blocking; the depth-nbo
  // trailing and back-substitution updates use `upd`, the nb-deep updates
  // inside an outer block are FP64 unless upd is UPD_EXACT_ALL.
  // tournament: tournament pivoting in the cluster panels (see launch_lu_panel).
  // lookahead (two-level blocking, nb-deep updates in FP64): the depth-nbo
  // update of the columns right of the next outer block runs on the side stream
  // while the next outer block's panels are factored; row exchanges of the
  // columns right of a block wait for its far phase.  The same operations in
  // the same order on every element: bit-identical results.
  bool lu_solve(const std::vector<LuDesc>& ds, int nb, Updates upd = UPD_FP64, unsigned char* pack = nullptr,
                size_t cap = 0, int* err = nullptr, int nbo = 0, int tournament = 0, int lookahead = 0);
  // Hermitian LDL^H without pivoting of the leading s x s block of every
  // problem (only its lower triangle is read), then the solve of the
  // right-hand-side columns s..ncols-1: panels of nb columns, trailing updates
  // on the lower triangle only (half the factorisation work of lu_solve),
  // back substitution as lu_solve.  upd: FP64 or exact tensor-core updates.
  bool ldl_solve(const std::vector<LuDesc>& ds, int nb, Updates upd = UPD_FP64, unsigned char* pack = nullptr,
                 size_t cap = 0, int* err = nullptr);
  void norm1(const std::vector<Norm1Desc>& ds) {
    if (ds.empty()) return;
    LaunchRec r;
    r.kind = K_NORM1;
    r.off = push_vec(ds);
    r.nprob = (int)ds.size();
    for (auto& d : ds) r.maxc = d.cols > r.maxc ? d.cols : r.maxc;
    recs_.push_back(r);
  }
  void frob2(const std::vector<Norm1Desc>& ds) {
    if (ds.empty()) return;
    LaunchRec r;
    r.kind = K_FROB2;
    r.off = push_vec(ds);
    r.nprob = (int)ds.size();
    for (auto& d : ds) r.maxc = d.cols > r.maxc ? d.cols : r.maxc;
    recs_.push_back(r);
  }
  void eig(const std::vector<EigDesc>& ds) {
    if (ds.empty()) return;
    LaunchRec r;
    r.kind = K_EIG;
    r.off = push_vec(ds);
    r.nprob = (int)ds.size();
    recs_.push_back(r);
  }
  void trace(const std::vector<TraceDesc>& ds) {
    if (ds.empty()) return;
    LaunchRec r;
    r.kind = K_TRACE;
    r.off = push_vec(ds);
    r.nprob = (int)ds.size();
    recs_.push_back(r);
  }
  void check(double* na, double* nb, const double* nd, int* act, int* iters, int* conv, int nprob,
             double tol, int cap, int count) {
    LaunchRec r;
    r.kind = K_CHECK;
    r.p[0] = na; r.p[1] = nb; r.p[2] = (void*)nd; r.p[3] = act; r.p[4] = iters; r.p[5] = conv;
    r.nprob = nprob; r.tol = tol; r.cap = cap; r.count = count;
    recs_.push_back(r);
  }
  void fill(int* p, int n, int v) {
    LaunchRec r;
    r.kind = K_FILL;
    r.p[0] = p; r.nprob = n; r.ival = v;
    recs_.push_back(r);
  }
  void memset0(void* p, size_t bytes) {
    LaunchRec r;
    r.kind = K_MEMSET;
    r.p[0] = p; r.bytes = bytes;
    recs_.push_back(r);
  }

  cudaError_t upload(cudaStream_t st);
  cudaError_t run(cudaStream_t st, long long* nlaunch, Prof* prof = nullptr);
  // Capture run() into a graph on first use, then replay it.
  cudaError_t replay(cudaStream_t st, long long* nlaunch);
  // run() or replay(): with graphs allowed and no profiling, a plan whose
  // launch sequence repeats the previous upload's (or has a graph already)
  // is replayed from its graph, any other runs eagerly (a one-off structure
  // is not worth an instantiation).
  cudaError_t execute(cudaStream_t st, long long* nlaunch, Prof* prof, bool graphs) {
    if (!graphs || prof) return run(st, nlaunch, prof);
    if (exec_ || repeat_ || runs_ > 0) return replay(st, nlaunch);  // the second run of one upload too
    ++runs_;
    return run(st, nlaunch, nullptr);
  }
  bool empty() const { return recs_.empty(); }

 private:
  bool oz_gemm_group(const std::vector<GemmDesc>& ds, unsigned char* pack, size_t cap, int* err, bool lu_label);
  void release();
  void destroy_graph();
  void fork() { LaunchRec r; r.kind = K_FORK; recs_.push_back(r); }
  void join() { LaunchRec r; r.kind = K_JOIN; recs_.push_back(r); }
  void to_side(size_t from) { for (size_t i = from; i < recs_.size(); ++i) recs_[i].side = 1; }
  std::vector<unsigned char> host_;
  std::vector<LaunchRec> recs_;
  cudaStream_t side_ = nullptr;  // created by upload() for plans that fork
  cudaEvent_t fork_ev_ = nullptr, join_ev_ = nullptr;
  unsigned char* dev_ = nullptr;
  size_t devcap_ = 0;
  cudaGraphExec_t exec_ = nullptr;
  long long graph_kernels_ = 0;
  int var_sq_ = -1, var_up_ = -1;
  size_t graph_sig_ = 0;  // signature of the launch sequence the graph was captured from
  size_t last_sig_ = 0;   // signature of the previous upload
  bool repeat_ = false;   // this upload repeats the previous one's launch sequence
  int runs_ = 0;          // eager runs since the last upload
  size_t signature() const;
};

}  // namespace ss
