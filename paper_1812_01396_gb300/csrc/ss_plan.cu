// Plan recording, upload, eager run and CUDA-graph replay.
#include "ss_plan.h"

#include <algorithm>

namespace ss {

void Plan::lu_solve(const std::vector<LuDesc>& ds, int nb) {
  if (ds.empty()) return;
  const size_t off = push_vec(ds);
  const int np = (int)ds.size();
  int smax = 0;
  for (auto& d : ds) smax = std::max(smax, d.s);
  if (nb <= 0) nb = lu_panel_width(smax);
  // forward: panels left to right
  for (int k0 = 0; k0 < smax; k0 += nb) {
    LaunchRec r;
    r.kind = K_LU_PANEL;
    r.off = off; r.nprob = np; r.k0 = k0; r.nb = nb; r.maxc = smax;
    recs_.push_back(r);
    int maxc = 0;
    std::vector<GemmDesc> g;
    for (auto& d : ds) {
      if (k0 >= d.s) continue;
      const int nbw = std::min(nb, d.s - k0);
      maxc = std::max(maxc, d.ncols - nbw);
      const int m = d.s - k0 - nbw, n = d.ncols - k0 - nbw;
      if (m <= 0 || n <= 0) continue;
      GemmDesc q{};
      q.m = m; q.n = n; q.k = nbw;
      q.a.p = d.w + (size_t)(k0 + nbw) * d.ldw + k0; q.a.ld = d.ldw;
      q.b.p = d.w + (size_t)k0 * d.ldw + k0 + nbw; q.b.ld = d.ldw;
      q.c = d.w + (size_t)(k0 + nbw) * d.ldw + k0 + nbw; q.ldc = d.ldw;
      q.alpha = make_double2(-1.0, 0.0); q.beta = make_double2(1.0, 0.0);
      q.active = d.active;
      g.push_back(q);
    }
    LaunchRec rr;
    rr.kind = K_LU_ROW;
    rr.off = off; rr.nprob = np; rr.k0 = k0; rr.nb = nb; rr.maxc = maxc;
    recs_.push_back(rr);
    gemm(g);
  }
  // backward substitution on the right-hand sides: panels right to left
  int maxrhs = 0;
  for (auto& d : ds) maxrhs = std::max(maxrhs, d.ncols - d.s);
  if (maxrhs <= 0) return;
  const int last = ((smax - 1) / nb) * nb;
  for (int k0 = last; k0 >= 0; k0 -= nb) {
    LaunchRec r;
    r.kind = K_LU_BACK;
    r.off = off; r.nprob = np; r.k0 = k0; r.nb = nb; r.maxc = maxrhs;
    recs_.push_back(r);
    if (k0 == 0) break;
    std::vector<GemmDesc> g;
    for (auto& d : ds) {
      if (k0 >= d.s || d.ncols <= d.s) continue;
      const int nbw = std::min(nb, d.s - k0);
      GemmDesc q{};
      q.m = k0; q.n = d.ncols - d.s; q.k = nbw;
      q.a.p = d.w + k0; q.a.ld = d.ldw;
      q.b.p = d.w + (size_t)k0 * d.ldw + d.s; q.b.ld = d.ldw;
      q.c = d.w + d.s; q.ldc = d.ldw;
      q.alpha = make_double2(-1.0, 0.0); q.beta = make_double2(1.0, 0.0);
      q.active = d.active;
      g.push_back(q);
    }
    gemm(g);
  }
}

void Plan::destroy_graph() {
  if (exec_) cudaGraphExecDestroy(exec_);
  exec_ = nullptr;
  graph_kernels_ = 0;
}

void Plan::release() {
  destroy_graph();
  if (dev_) cudaFree(dev_);
  dev_ = nullptr;
  devcap_ = 0;
}

cudaError_t Plan::upload(cudaStream_t st) {
  destroy_graph();
  const size_t need = host_.size() ? host_.size() : 16;
  if (need > devcap_) {
    if (dev_) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return e;
      cudaFree(dev_);
      dev_ = nullptr;
    }
    size_t cap = std::max<size_t>(need, 1 << 16);
    cudaError_t e = cudaMalloc(&dev_, cap);
    if (e != cudaSuccess) { dev_ = nullptr; devcap_ = 0; return e; }
    devcap_ = cap;
  }
  if (host_.empty()) return cudaSuccess;
  return cudaMemcpyAsync(dev_, host_.data(), host_.size(), cudaMemcpyHostToDevice, st);
}

static double gemm_flops(const LaunchRec& r, const std::vector<unsigned char>& host, const Prof* prof) {
  const GemmDesc* g = reinterpret_cast<const GemmDesc*>(host.data() + r.off);
  double f = 0.0;
  for (int i = 0; i < r.nprob; ++i) {
    if (g[i].active && prof->act_host) {
      const long idx = g[i].active - prof->act_dev;
      if (idx >= 0 && idx < prof->nact && !prof->act_host[idx]) continue;
    }
    f += 8.0 * g[i].m * (double)g[i].n * g[i].k;
  }
  return f;
}

cudaError_t Plan::run(cudaStream_t st, long long* nlaunch, Prof* prof) {
  long long n = 0;
  for (const LaunchRec& r : recs_) {
    Prof::Rec pr{};
    if (prof && r.kind != K_MEMSET) {
      pr.kind = r.kind;
      pr.flops = r.kind == K_GEMM ? gemm_flops(r, host_, prof) : 0.0;
      cudaEventCreate(&pr.a);
      cudaEventCreate(&pr.b);
      cudaEventRecord(pr.a, st);
    }
    unsigned char* d = dev_ + r.off;
    const int* t = reinterpret_cast<const int*>(dev_ + r.toff);
    switch (r.kind) {
      case K_GEMM: launch_zgemm((const GemmDesc*)d, t, r.nprob, r.tiles, st); ++n; break;
      case K_FORM: launch_zform((const FormDesc*)d, t, r.nprob, r.tiles, st); ++n; break;
      case K_LU_PANEL: launch_lu_panel((const LuDesc*)d, r.nprob, r.k0, r.nb, r.maxc, st); ++n; break;
      case K_LU_ROW:
        if (r.maxc > 0) { launch_lu_rowblock((const LuDesc*)d, r.nprob, r.k0, r.nb, r.maxc, st); ++n; }
        break;
      case K_LU_BACK: launch_lu_backsub_diag((const LuDesc*)d, r.nprob, r.k0, r.nb, r.maxc, st); ++n; break;
      case K_NORM1: launch_norm1((const Norm1Desc*)d, r.nprob, r.maxc, st); ++n; break;
      case K_TRACE: launch_trace((const TraceDesc*)d, r.nprob, st); ++n; break;
      case K_CHECK:
        launch_decim_check((double*)r.p[0], (double*)r.p[1], (const double*)r.p[2], (int*)r.p[3],
                           (int*)r.p[4], (int*)r.p[5], r.nprob, r.tol, r.cap, r.count, st);
        ++n;
        break;
      case K_FILL: launch_fill_i32((int*)r.p[0], r.nprob, r.ival, st); ++n; break;
      case K_MEMSET: {
        cudaError_t e = cudaMemsetAsync(r.p[0], 0, r.bytes, st);
        if (e != cudaSuccess) return e;
        break;
      }
    }
    if (prof && r.kind != K_MEMSET) {
      cudaEventRecord(pr.b, st);
      prof->recs.push_back(pr);
    }
  }
  if (nlaunch) *nlaunch += n;
  return cudaGetLastError();
}

cudaError_t Plan::replay(cudaStream_t st, long long* nlaunch) {
  if (!exec_) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    long long n = 0;
    cudaError_t er = run(st, &n);
    e = cudaStreamEndCapture(st, &g);
    if (er != cudaSuccess) { if (g) cudaGraphDestroy(g); return er; }
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return e; }
    e = cudaGraphInstantiate(&exec_, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { exec_ = nullptr; return e; }
    graph_kernels_ = n;
  }
  cudaError_t e = cudaGraphLaunch(exec_, st);
  if (nlaunch) *nlaunch += graph_kernels_;
  return e;
}

}  // namespace ss
