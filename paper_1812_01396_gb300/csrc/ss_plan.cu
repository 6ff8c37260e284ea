// Plan recording, upload, eager run and CUDA-graph replay.
#include "ss_plan.h"

#include <algorithm>
#include <map>
#include <tuple>

namespace ss {

namespace {
thread_local long long g_host_calls = 0;
}  // namespace
long long host_launch_calls() { return g_host_calls; }

namespace {
struct OpKey {
  const void* p; const void* s; double er, ei; int ld, trans, rows, k, role;
  bool operator<(const OpKey& o) const {
    return std::tie(p, s, er, ei, ld, trans, rows, k, role) <
           std::tie(o.p, o.s, o.er, o.ei, o.ld, o.trans, o.rows, o.k, o.role);
  }
};
size_t al1k(size_t x) { return (x + 1023) & ~size_t(1023); }
}  // namespace

namespace {
size_t oz_operand_bytes(int rows, int vecs, int k) {
  OzShape sh;
  oz_plan(k, &sh);
  return al1k((size_t)rows * sh.S * sh.w * 2) + al1k((size_t)vecs * sizeof(unsigned long long));
}
}  // namespace

size_t Plan::oz_pack_bytes(const std::vector<GemmDesc>& ds) {
  std::map<OpKey, int> seen;
  size_t tot = 0;
  for (auto& g : ds) {
    OpKey ka{g.a.p, g.a.s, g.a.e.x, g.a.e.y, g.a.ld, g.a.trans, g.m, g.k, 0};
    OpKey kb{g.b.p, g.b.s, g.b.e.x, g.b.e.y, g.b.ld, g.b.trans, 2 * g.n, g.k, 1};
    if (!seen.count(ka)) { seen[ka] = 1; tot += oz_operand_bytes(g.m, g.m, g.k); }
    if (!seen.count(kb)) { seen[kb] = 1; tot += oz_operand_bytes(2 * g.n, g.n, g.k); }
  }
  return tot;
}

bool Plan::oz_gemm(const std::vector<GemmDesc>& ds, unsigned char* pack, size_t cap, int* err, bool lu_label) {
  if (ds.empty()) return true;
  if (oz_pack_bytes(ds) <= cap) return oz_gemm_group(ds, pack, cap, err, lu_label);
  // the digit slices of the whole group do not fit: consecutive chunks that
  // do, one after the other (the GEMMs of a group are independent)
  std::vector<GemmDesc> chunk;
  std::map<OpKey, int> seen;
  size_t bytes = 0;
  for (const GemmDesc& g : ds) {
    const OpKey ka{g.a.p, g.a.s, g.a.e.x, g.a.e.y, g.a.ld, g.a.trans, g.m, g.k, 0};
    const OpKey kb{g.b.p, g.b.s, g.b.e.x, g.b.e.y, g.b.ld, g.b.trans, 2 * g.n, g.k, 1};
    const size_t need = (seen.count(ka) ? 0 : oz_operand_bytes(g.m, g.m, g.k)) +
                        (seen.count(kb) ? 0 : oz_operand_bytes(2 * g.n, g.n, g.k));
    if (bytes + need > cap) {
      if (chunk.empty()) return false;  // a single GEMM does not fit
      if (!oz_gemm_group(chunk, pack, cap, err, lu_label)) return false;
      chunk.clear();
      seen.clear();
      bytes = oz_operand_bytes(g.m, g.m, g.k) + oz_operand_bytes(2 * g.n, g.n, g.k);
    } else {
      bytes += need;
    }
    seen[ka] = 1;
    seen[kb] = 1;
    chunk.push_back(g);
  }
  return oz_gemm_group(chunk, pack, cap, err, lu_label);
}

bool Plan::oz_gemm_group(const std::vector<GemmDesc>& ds, unsigned char* pack, size_t cap, int* err,
                         bool lu_label) {
  std::map<OpKey, int> index;
  std::vector<OzPackDesc> pk;
  std::vector<size_t> dbytes;  // digit bytes of each distinct operand
  std::vector<int> amap(ds.size()), bmap(ds.size());
  std::vector<OzShape> shapes(ds.size());
  size_t nmax = 0;  // maxima of all operands, one contiguous array
  for (size_t i = 0; i < ds.size(); ++i) {
    const GemmDesc& g = ds[i];
    oz_plan(g.k, &shapes[i]);
    const OzShape& sh = shapes[i];
    if (sh.npass > OZ_MAXPASS) return false;
    for (int role = 0; role < 2; ++role) {
      const Operand& o = role == 0 ? g.a : g.b;
      const int rows = role == 0 ? g.m : 2 * g.n;
      const int vecs = role == 0 ? g.m : g.n;
      OpKey key{o.p, o.s, o.e.x, o.e.y, o.ld, o.trans, rows, g.k, role};
      auto it = index.find(key);
      int mi;
      if (it == index.end()) {
        OzPackDesc d{};
        d.x = o.p; d.s = o.s; d.e = o.e; d.ld = o.ld; d.trans = o.trans; d.role = role;
        d.rows = rows; d.k = g.k; d.w = sh.w; d.S = sh.S; d.beta_bits = sh.beta;
        d.maxb = reinterpret_cast<unsigned long long*>(pack) + nmax;
        d.active = g.active;
        nmax += (size_t)vecs;
        mi = (int)pk.size();
        pk.push_back(d);
        dbytes.push_back(al1k((size_t)rows * sh.S * sh.w * 2));
        index[key] = mi;
      } else {
        mi = it->second;
      }
      (role == 0 ? amap : bmap)[i] = mi;
    }
  }
  // layout: [maxima | digit slices of each operand, 1 KB aligned]
  size_t used = al1k(nmax * sizeof(unsigned long long));
  std::vector<CUtensorMap> maps(pk.size());
  for (size_t q = 0; q < pk.size(); ++q) {
    if (used + dbytes[q] > cap) return false;
    pk[q].out = reinterpret_cast<__nv_bfloat16*>(pack + used);
    if (encode_kmajor_map(&maps[q], pack + used, pk[q].rows, pk[q].S * pk[q].w,
                          pk[q].role == 0 ? oz_box_rows_a() : oz_box_rows_b()) != cudaSuccess)
      return false;
    used += dbytes[q];
  }
  // maxima (zeroed first, one memset for the group), then digit slices
  {
    memset0(pack, nmax * sizeof(unsigned long long));
    std::vector<int> start(pk.size());
    int tot = 0;
    for (size_t i = 0; i < pk.size(); ++i) {
      start[i] = tot;
      tot += oz_scale_tiles(pk[i]);
    }
    const size_t off = push_vec(pk);
    LaunchRec r;
    r.kind = K_OZSCALE; r.off = off; r.toff = push_vec(start); r.nprob = (int)pk.size(); r.tiles = tot;
    recs_.push_back(r);
    std::vector<int> start2(pk.size());
    int tot2 = 0;
    for (size_t i = 0; i < pk.size(); ++i) { start2[i] = tot2; tot2 += oz_pack_tiles(pk[i]); }
    LaunchRec r2;
    r2.kind = K_OZPACK; r2.off = off; r2.toff = push_vec(start2); r2.nprob = (int)pk.size(); r2.tiles = tot2;
    recs_.push_back(r2);
  }
  std::vector<OzDesc> ods(ds.size());
  std::vector<int> start(ds.size());
  int tot = 0;
  for (size_t i = 0; i < ds.size(); ++i) {
    const GemmDesc& g = ds[i];
    const OzShape& sh = shapes[i];
    OzDesc t{};
    t.m = g.m; t.n2 = 2 * g.n; t.w = sh.w; t.kc = g.k; t.beta_bits = sh.beta; t.npass = sh.npass;
    for (int p = 0; p < sh.npass; ++p) { t.pd[p] = sh.pd[p]; t.pt0[p] = sh.pt0[p]; t.pnp[p] = sh.pnp[p]; }
    t.mA = pk[amap[i]].maxb;
    t.mB = pk[bmap[i]].maxb;
    t.c = g.c; t.ldc = g.ldc; t.cmode = g.cmode; t.alpha = g.alpha; t.beta = g.beta;
    t.cs = g.cs; t.ch = g.ch; t.ce = g.ce; t.ldcf = g.ldcf; t.active = g.active; t.lower = g.lower;
    ods[i] = t;
    start[i] = tot;
    tot += oz_tiles(t.m, t.n2);
  }
  const size_t doff = push(nullptr, ods.size() * sizeof(OzDesc), 64);
  const size_t moff = push_vec(maps, 64);
  for (size_t i = 0; i < ds.size(); ++i) {
    ods[i].ta_off = (long long)(moff + (size_t)amap[i] * sizeof(CUtensorMap) - doff);
    ods[i].tb_off = (long long)(moff + (size_t)bmap[i] * sizeof(CUtensorMap) - doff);
  }
  std::memcpy(host_.data() + doff, ods.data(), ods.size() * sizeof(OzDesc));
  LaunchRec r;
  r.kind = lu_label ? K_OZGEMM_LU : K_OZGEMM; r.off = doff; r.toff = push_vec(start); r.nprob = (int)ds.size();
  r.tiles = tot;
  r.p[0] = err;
  recs_.push_back(r);
  return true;
}

size_t Plan::tc_pack_bytes(const std::vector<GemmDesc>& ds, int mode) {
  std::map<OpKey, int> seen;
  size_t tot = 0;
  for (auto& g : ds) {
    const int kp = tc_kp(g.k, mode);
    OpKey ka{g.a.p, g.a.s, g.a.e.x, g.a.e.y, g.a.ld, g.a.trans, g.m, g.k, 0};
    OpKey kb{g.b.p, g.b.s, g.b.e.x, g.b.e.y, g.b.ld, g.b.trans, 2 * g.n, g.k, 1};
    if (!seen.count(ka)) { seen[ka] = 1; tot += al1k((size_t)g.m * kp * 2); }
    if (!seen.count(kb)) { seen[kb] = 1; tot += al1k((size_t)2 * g.n * kp * 2); }
  }
  return tot;
}

bool Plan::tc_gemm(const std::vector<GemmDesc>& ds, int mode, unsigned char* pack, size_t cap, int* err) {
  if (ds.empty()) return true;
  std::map<OpKey, int> index;   // operand -> position in pa / pb
  std::vector<PackDesc> pa, pb;
  std::vector<CUtensorMap> maps;
  std::vector<int> map_of_a, map_of_b;
  std::vector<int> amap(ds.size()), bmap(ds.size());
  size_t used = 0;
  for (size_t i = 0; i < ds.size(); ++i) {
    const GemmDesc& g = ds[i];
    const int kp = tc_kp(g.k, mode);
    for (int role = 0; role < 2; ++role) {
      const Operand& o = role == 0 ? g.a : g.b;
      const int rows = role == 0 ? g.m : 2 * g.n;
      OpKey key{o.p, o.s, o.e.x, o.e.y, o.ld, o.trans, rows, g.k, role};
      auto it = index.find(key);
      int mi;
      if (it == index.end()) {
        const size_t bytes = al1k((size_t)rows * kp * 2);
        if (used + bytes > cap) return false;
        PackDesc d{};
        d.x = o.p; d.s = o.s; d.e = o.e; d.ld = o.ld; d.trans = o.trans;
        d.rows = rows; d.k = g.k; d.kp = kp;
        d.out = reinterpret_cast<__nv_bfloat16*>(pack + used);
        d.active = g.active;
        CUtensorMap m;
        if (encode_kmajor_map(&m, pack + used, rows, kp, role == 0 ? tc_box_rows_a() : tc_box_rows_b()) !=
            cudaSuccess)
          return false;
        used += bytes;
        mi = (int)maps.size();
        maps.push_back(m);
        (role == 0 ? pa : pb).push_back(d);
        index[key] = mi;
      } else {
        mi = it->second;
      }
      (role == 0 ? amap : bmap)[i] = mi;
    }
  }
  // pack launches
  for (int role = 0; role < 2; ++role) {
    std::vector<PackDesc>& v = role == 0 ? pa : pb;
    std::vector<int> start(v.size());
    int tot = 0;
    for (size_t i = 0; i < v.size(); ++i) { start[i] = tot; tot += pack_tiles(v[i].rows, v[i].kp); }
    LaunchRec r;
    r.kind = role == 0 ? K_PACK_A : K_PACK_B;
    r.off = push_vec(v);
    r.toff = push_vec(start);
    r.nprob = (int)v.size();
    r.tiles = tot;
    r.ival = mode;
    recs_.push_back(r);
  }
  // GEMM descriptors followed by their tensor maps (64-byte aligned)
  std::vector<TcDesc> tds(ds.size());
  std::vector<int> start(ds.size());
  int tot = 0;
  for (size_t i = 0; i < ds.size(); ++i) {
    const GemmDesc& g = ds[i];
    TcDesc t{};
    t.m = g.m; t.n2 = 2 * g.n; t.kp = tc_kp(g.k, mode); t.kc = g.k;
    t.c = g.c; t.ldc = g.ldc; t.cmode = g.cmode; t.alpha = g.alpha; t.beta = g.beta;
    t.cs = g.cs; t.ch = g.ch; t.ce = g.ce; t.ldcf = g.ldcf; t.active = g.active;
    tds[i] = t;
    start[i] = tot;
    tot += tc_tiles(t.m, t.n2);
  }
  const size_t doff = push(nullptr, tds.size() * sizeof(TcDesc), 64);
  const size_t moff = push_vec(maps, 64);
  for (size_t i = 0; i < ds.size(); ++i) {
    tds[i].ta_off = (long long)(moff + (size_t)amap[i] * sizeof(CUtensorMap) - doff);
    tds[i].tb_off = (long long)(moff + (size_t)bmap[i] * sizeof(CUtensorMap) - doff);
  }
  std::memcpy(host_.data() + doff, tds.data(), tds.size() * sizeof(TcDesc));
  LaunchRec r;
  r.kind = K_TCGEMM;
  r.off = doff;
  r.toff = push_vec(start);
  r.nprob = (int)ds.size();
  r.tiles = tot;
  r.p[0] = err;
  recs_.push_back(r);
  return true;
}

bool Plan::lu_solve(const std::vector<LuDesc>& ds, int nb, Updates upd, unsigned char* pack, size_t cap, int* err,
                    int nbo, int tournament, int lookahead) {
  if (ds.empty()) return true;
  bool ok = true;
  auto update = [&](const std::vector<GemmDesc>& g) {
    if (upd == UPD_EXACT_TC || upd == UPD_EXACT_ALL || upd == UPD_EXACT_FAR) ok = ok && oz_gemm(g, pack, cap, err, true);
    else gemm(g, true);
  };
  // the nb-deep updates inside an outer block (two-level blocking)
  auto inner_update = [&](const std::vector<GemmDesc>& g) {
    if (upd == UPD_EXACT_ALL) ok = ok && oz_gemm(g, pack, cap, err, true);
    else gemm(g, true);
  };
  // the outer block's rows on the columns right of it (nb deep, wide)
  auto far_update = [&](const std::vector<GemmDesc>& g) {
    if (upd == UPD_EXACT_ALL || upd == UPD_EXACT_FAR) ok = ok && oz_gemm(g, pack, cap, err, true);
    else gemm(g, true);
  };
  const int np = (int)ds.size();
  int smax = 0;
  for (auto& d : ds) smax = std::max(smax, d.s);
  if (nb <= 0) nb = lu_panel_width(smax);
  if (nbo > 0 && (nbo <= nb || nbo % nb != 0)) nbo = 0;
  const size_t off = push_vec(ds);
  // C -= A B with A at (ar, ac), B at (br, bc), C at (cr, cc) of the problem's W
  auto upd_desc = [](const LuDesc& d, int m, int n, int k, int ar, int ac, int br, int bc, int cr, int cc) {
    GemmDesc q{};
    q.m = m; q.n = n; q.k = k;
    q.a.p = d.w + (size_t)ar * d.ldw + ac; q.a.ld = d.ldw;
    q.b.p = d.w + (size_t)br * d.ldw + bc; q.b.ld = d.ldw;
    q.c = d.w + (size_t)cr * d.ldw + cc; q.ldc = d.ldw;
    q.alpha = make_double2(-1.0, 0.0); q.beta = make_double2(1.0, 0.0);
    q.active = d.active;
    return q;
  };
  auto rowblock = [&](int k0, int far, int maxc) {
    LaunchRec rr;
    rr.kind = K_LU_ROW;
    rr.off = off; rr.nprob = np; rr.k0 = k0; rr.nb = nb; rr.nbo = nbo; rr.ival = far; rr.maxc = maxc;
    rr.cap = smax;  // rows of the largest block (the exchange gather's staging)
    recs_.push_back(rr);
  };
  auto panel = [&](int k0) {
    LaunchRec r;
    r.kind = K_LU_PANEL;
    r.off = off; r.nprob = np; r.k0 = k0; r.nb = nb; r.maxc = smax; r.ival = tournament;
    recs_.push_back(r);
  };
  if (nbo <= 0) {
    // forward: panels left to right
    for (int k0 = 0; k0 < smax; k0 += nb) {
      panel(k0);
      int maxc = 0;
      std::vector<GemmDesc> g;
      for (auto& d : ds) {
        if (k0 >= d.s) continue;
        const int nbw = std::min(nb, d.s - k0);
        maxc = std::max(maxc, d.ncols - nbw);
        const int m = d.s - k0 - nbw, n = d.ncols - k0 - nbw;
        if (m <= 0 || n <= 0) continue;
        g.push_back(upd_desc(d, m, n, nbw, k0 + nbw, k0, k0, k0 + nbw, k0 + nbw, k0 + nbw));
      }
      rowblock(k0, 0, maxc);
      update(g);
    }
  } else {
    // lookahead needs the nb-deep updates off the packing buffer (FP64), which
    // the side stream's exact update may be using meanwhile
    const bool la = lookahead && upd != UPD_EXACT_ALL;
    bool forked = false;  // a side-stream trailing update not yet joined
    for (int K0 = 0; K0 < smax; K0 += nbo) {
      const int kend = std::min(K0 + nbo, smax);
      // nb-wide steps inside the outer block (with lookahead: row exchanges on
      // the block's own columns only; they touch nothing the side stream writes)
      for (int k0 = K0; k0 < kend; k0 += nb) {
        panel(k0);
        int maxc = 0;
        std::vector<GemmDesc> g;
        for (auto& d : ds) {
          if (k0 >= d.s) continue;
          const int nbw = std::min(nb, d.s - k0), K1 = std::min(K0 + nbo, d.s);
          maxc = std::max(maxc, la ? K1 - nbw - K0 : d.ncols - nbw);
          const int m = d.s - k0 - nbw, n = K1 - k0 - nbw;
          if (m <= 0 || n <= 0) continue;
          g.push_back(upd_desc(d, m, n, nbw, k0 + nbw, k0, k0, k0 + nbw, k0 + nbw, k0 + nbw));
        }
        rowblock(k0, la ? 2 : 0, maxc);
        inner_update(g);
      }
      if (forked) {  // the columns right of this block are up to date from here on
        join();
        forked = false;
      }
      // the block's rows on the columns right of it (with lookahead: the row
      // exchanges of all the block's panels on those columns first)
      if (la) {
        int maxc = 0;
        for (auto& d : ds)
          if (K0 < d.s) maxc = std::max(maxc, d.ncols - std::min(K0 + nbo, d.s));
        rowblock(K0, 3, maxc);
      }
      for (int k0 = K0; k0 < kend; k0 += nb) {
        int maxc = 0;
        std::vector<GemmDesc> g;
        for (auto& d : ds) {
          if (k0 >= d.s) continue;
          const int nbw = std::min(nb, d.s - k0), K1 = std::min(K0 + nbo, d.s);
          maxc = std::max(maxc, d.ncols - K1);
          const int m = K1 - k0 - nbw, n = d.ncols - K1;
          if (m <= 0 || n <= 0) continue;
          g.push_back(upd_desc(d, m, n, nbw, k0 + nbw, k0, k0, K1, k0 + nbw, K1));
        }
        rowblock(k0, 1, maxc);
        far_update(g);
      }
      // one trailing update of depth nbo; with lookahead split into the next
      // outer block's columns (now) and the columns right of it (side stream)
      std::vector<GemmDesc> g, gw;
      for (auto& d : ds) {
        if (K0 >= d.s) continue;
        const int K1 = std::min(K0 + nbo, d.s);
        const int m = d.s - K1, n = d.ncols - K1;
        if (m <= 0 || n <= 0) continue;
        if (!la) {
          g.push_back(upd_desc(d, m, n, K1 - K0, K1, K0, K0, K1, K1, K1));
          continue;
        }
        const int K2 = std::min(K1 + nbo, d.s);
        g.push_back(upd_desc(d, m, K2 - K1, K1 - K0, K1, K0, K0, K1, K1, K1));
        if (d.ncols > K2) gw.push_back(upd_desc(d, m, d.ncols - K2, K1 - K0, K1, K0, K0, K2, K1, K2));
      }
      update(g);
      if (!gw.empty()) {
        fork();
        const size_t mark = recs_.size();
        update(gw);
        to_side(mark);
        forked = true;
      }
    }
    if (forked) join();
  }
  // backward substitution on the right-hand sides: panels right to left
  int maxrhs = 0;
  for (auto& d : ds) maxrhs = std::max(maxrhs, d.ncols - d.s);
  if (maxrhs <= 0) return ok;
  const int last = ((smax - 1) / nb) * nb;
  for (int k0 = last; k0 >= 0; k0 -= nb) {
    LaunchRec r;
    r.kind = K_LU_BACK;
    r.off = off; r.nprob = np; r.k0 = k0; r.nb = nb; r.maxc = maxrhs;
    recs_.push_back(r);
    if (k0 == 0) break;
    std::vector<GemmDesc> g;
    if (nbo <= 0) {
      for (auto& d : ds) {
        if (k0 >= d.s || d.ncols <= d.s) continue;
        const int nbw = std::min(nb, d.s - k0);
        g.push_back(upd_desc(d, k0, d.ncols - d.s, nbw, 0, k0, k0, d.s, 0, d.s));
      }
      update(g);
      continue;
    }
    const int K0 = (k0 / nbo) * nbo;
    if (k0 > K0) {
      // rows of the outer block above this panel, FP64
      for (auto& d : ds) {
        if (k0 >= d.s || d.ncols <= d.s) continue;
        const int nbw = std::min(nb, d.s - k0);
        g.push_back(upd_desc(d, k0 - K0, d.ncols - d.s, nbw, K0, k0, k0, d.s, K0, d.s));
      }
      inner_update(g);
    } else {
      // every row above the outer block, depth nbo
      for (auto& d : ds) {
        if (K0 >= d.s || d.ncols <= d.s) continue;
        const int K1 = std::min(K0 + nbo, d.s);
        g.push_back(upd_desc(d, K0, d.ncols - d.s, K1 - K0, 0, K0, K0, d.s, 0, d.s));
      }
      update(g);
    }
  }
  return ok;
}

bool Plan::ldl_solve(const std::vector<LuDesc>& ds, int nb, Updates upd, unsigned char* pack, size_t cap, int* err) {
  if (ds.empty()) return true;
  bool ok = true;
  auto update = [&](const std::vector<GemmDesc>& g) {
    if (upd == UPD_EXACT_TC || upd == UPD_EXACT_ALL) ok = ok && oz_gemm(g, pack, cap, err, true);
    else gemm(g, true);
  };
  const int np = (int)ds.size();
  int smax = 0, maxrhs = 0;
  for (auto& d : ds) { smax = std::max(smax, d.s); maxrhs = std::max(maxrhs, d.ncols - d.s); }
  if (nb <= 0) nb = 16;
  nb = std::min(nb, 32);
  const size_t off = push_vec(ds);
  auto udesc = [](const LuDesc& d, int m, int n, int k, int ar, int ac, int br, int bc, int cr, int cc) {
    GemmDesc q{};
    q.m = m; q.n = n; q.k = k;
    q.a.p = d.w + (size_t)ar * d.ldw + ac; q.a.ld = d.ldw;
    q.b.p = d.w + (size_t)br * d.ldw + bc; q.b.ld = d.ldw;
    q.c = d.w + (size_t)cr * d.ldw + cc; q.ldc = d.ldw;
    q.alpha = make_double2(-1.0, 0.0); q.beta = make_double2(1.0, 0.0);
    q.active = d.active;
    return q;
  };
  for (int k0 = 0; k0 < smax; k0 += nb) {
    LaunchRec r;
    r.kind = K_LU_HPANEL;
    r.off = off; r.nprob = np; r.k0 = k0; r.nb = nb; r.maxc = smax;
    recs_.push_back(r);
    if (maxrhs > 0) {  // B1 = L11^-1 B1 on the right-hand sides (no row exchanges)
      LaunchRec rr;
      rr.kind = K_LU_ROW;
      rr.off = off; rr.nprob = np; rr.k0 = k0; rr.nb = nb; rr.nbo = -1; rr.ival = 1; rr.maxc = maxrhs;
      recs_.push_back(rr);
    }
    std::vector<GemmDesc> g;
    for (auto& d : ds) {
      if (k0 >= d.s) continue;
      const int nbw = std::min(nb, d.s - k0);
      const int m = d.s - k0 - nbw;
      if (m <= 0) continue;
      GemmDesc q = udesc(d, m, m, nbw, k0 + nbw, k0, k0, k0 + nbw, k0 + nbw, k0 + nbw);
      q.lower = 1;  // A22 -= L21 U12 on the lower triangle
      g.push_back(q);
      if (d.ncols > d.s) g.push_back(udesc(d, m, d.ncols - d.s, nbw, k0 + nbw, k0, k0, d.s, k0 + nbw, d.s));
    }
    update(g);
  }
  if (maxrhs <= 0) return ok;
  // back substitution with U = D L^H (written by the panels), as in lu_solve
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
      g.push_back(udesc(d, k0, d.ncols - d.s, nbw, 0, k0, k0, d.s, 0, d.s));
    }
    update(g);
  }
  return ok;
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
  if (side_) cudaStreamDestroy(side_);
  if (fork_ev_) cudaEventDestroy(fork_ev_);
  if (join_ev_) cudaEventDestroy(join_ev_);
  side_ = nullptr;
  fork_ev_ = join_ev_ = nullptr;
}

// Hash of everything a captured launch depends on except the descriptor
// contents: the device buffer, and per launch its kind, grid sizes, offsets
// into the buffer, scalar and pointer arguments.
size_t Plan::signature() const {
  size_t h = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) { h = (h ^ v) * 1099511628211ull; };
  mix((unsigned long long)(uintptr_t)dev_);
  mix(recs_.size());
  for (const LaunchRec& r : recs_) {
    mix((unsigned long long)r.kind); mix(r.off); mix(r.toff); mix((unsigned)r.nprob); mix((unsigned)r.tiles);
    mix((unsigned)r.k0); mix((unsigned)r.nb); mix((unsigned)r.maxc); mix((unsigned)r.nbo);
    unsigned long long tb;
    std::memcpy(&tb, &r.tol, sizeof(tb));
    mix(tb); mix((unsigned)r.cap); mix((unsigned)r.count); mix((unsigned)r.ival); mix(r.bytes); mix((unsigned)r.side);
    for (int i = 0; i < 6; ++i) mix((unsigned long long)(uintptr_t)r.p[i]);
  }
  return h;
}

cudaError_t Plan::upload(cudaStream_t st) {
  if (!side_ && std::any_of(recs_.begin(), recs_.end(), [](const LaunchRec& r) { return r.kind == K_FORK; })) {
    cudaError_t e = cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork_ev_, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join_ev_, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  const size_t need = host_.size() ? host_.size() : 16;
  if (need > devcap_) {
    destroy_graph();
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
  const size_t sig = signature();
  repeat_ = sig == last_sig_;
  last_sig_ = sig;
  runs_ = 0;
  if (exec_ && sig != graph_sig_) destroy_graph();
  if (host_.empty()) return cudaSuccess;
  return cudaMemcpyAsync(dev_, host_.data(), host_.size(), cudaMemcpyHostToDevice, st);
}

static bool prof_active(const int* a, const Prof* prof) {
  if (!a || !prof->act_host) return true;
  const long idx = a - prof->act_dev;
  return !(idx >= 0 && idx < prof->nact && !prof->act_host[idx]);
}

static double oz_issued(const LaunchRec& r, const std::vector<unsigned char>& host, const Prof* prof) {
  const OzDesc* g = reinterpret_cast<const OzDesc*>(host.data() + r.off);
  double f = 0.0;
  for (int i = 0; i < r.nprob; ++i) {
    if (!prof_active(g[i].active, prof)) continue;
    int pairs = 0;
    for (int p = 0; p < g[i].npass; ++p) pairs += g[i].pnp[p];
    f += 2.0 * g[i].m * (double)g[i].n2 * (double)pairs * g[i].w;
  }
  return f;
}

static double gemm_flops(const LaunchRec& r, const std::vector<unsigned char>& host, const Prof* prof) {
  double f = 0.0;
  if (r.kind == K_GEMM || r.kind == K_GEMM32 || r.kind == K_GEMM_LU) {
    const GemmDesc* g = reinterpret_cast<const GemmDesc*>(host.data() + r.off);
    for (int i = 0; i < r.nprob; ++i)
      if (prof_active(g[i].active, prof))
        f += 8.0 * g[i].k * (g[i].lower ? 0.5 * g[i].m * (double)(g[i].n + 1) : g[i].m * (double)g[i].n);
  } else if (r.kind == K_OZGEMM || r.kind == K_OZGEMM_LU) {
    const OzDesc* g = reinterpret_cast<const OzDesc*>(host.data() + r.off);
    for (int i = 0; i < r.nprob; ++i)
      if (prof_active(g[i].active, prof))
        f += 8.0 * g[i].kc * (g[i].lower ? 0.5 * g[i].m * (double)(g[i].n2 / 2 + 1) : g[i].m * (double)(g[i].n2 / 2));
  } else if (r.kind == K_TCGEMM) {
    // algorithmic complex flops (8 m n k), not the split-term tensor flops
    const TcDesc* g = reinterpret_cast<const TcDesc*>(host.data() + r.off);
    for (int i = 0; i < r.nprob; ++i)
      if (prof_active(g[i].active, prof)) f += 8.0 * g[i].m * (double)(g[i].n2 / 2) * (double)g[i].kc;
  }
  return f;
}

cudaError_t Plan::run(cudaStream_t st, long long* nlaunch, Prof* prof) {
  long long n = 0;
  const cudaStream_t main_st = st;
  for (const LaunchRec& r : recs_) {
    if (r.kind == K_FORK || r.kind == K_JOIN) {
      cudaError_t e = r.kind == K_FORK ? cudaEventRecord(fork_ev_, main_st) : cudaEventRecord(join_ev_, side_);
      if (e == cudaSuccess)
        e = r.kind == K_FORK ? cudaStreamWaitEvent(side_, fork_ev_, 0) : cudaStreamWaitEvent(main_st, join_ev_, 0);
      if (e != cudaSuccess) return e;
      continue;
    }
    st = r.side ? side_ : main_st;
    Prof::Rec pr{};
    if (prof && r.kind != K_MEMSET) {
      pr.kind = r.kind;
      pr.flops = (r.kind == K_GEMM || r.kind == K_TCGEMM || r.kind == K_GEMM32 || r.kind == K_OZGEMM ||
                  r.kind == K_GEMM_LU || r.kind == K_OZGEMM_LU)
                     ? gemm_flops(r, host_, prof)
                     : 0.0;
      pr.issued = (r.kind == K_OZGEMM || r.kind == K_OZGEMM_LU) ? oz_issued(r, host_, prof) : 0.0;
      cudaEventCreate(&pr.a);
      cudaEventCreate(&pr.b);
      cudaEventRecord(pr.a, st);
    }
    unsigned char* d = dev_ + r.off;
    const int* t = reinterpret_cast<const int*>(dev_ + r.toff);
    switch (r.kind) {
      case K_GEMM:
      case K_GEMM_LU: launch_zgemm((const GemmDesc*)d, t, r.nprob, r.tiles, st, r.ival); ++n; break;
      case K_OZSCALE: launch_oz_scale((const OzPackDesc*)d, t, r.nprob, r.tiles, st); ++n; break;
      case K_OZPACK: launch_oz_pack((const OzPackDesc*)d, t, r.nprob, r.tiles, st); ++n; break;
      case K_OZGEMM:
      case K_OZGEMM_LU: {
        cudaError_t e = launch_oz_gemm((const OzDesc*)d, t, r.nprob, r.tiles, (int*)r.p[0], st);
        if (e != cudaSuccess) return e;
        ++n;
        break;
      }
      case K_FORM: launch_zform((const FormDesc*)d, t, r.nprob, r.tiles, st); ++n; break;
      case K_LU_PANEL: launch_lu_panel((const LuDesc*)d, r.nprob, r.k0, r.nb, r.maxc, st, r.ival); ++n; break;
      case K_LU_HPANEL:
        launch_herm_panel((const LuDesc*)d, r.nprob, r.k0, r.nb, r.maxc, st);
        n += (r.maxc - r.k0 - r.nb > 0) ? 2 : 1;
        break;
      case K_LU_ROW:
        if (r.maxc > 0) {
          launch_lu_rowblock((const LuDesc*)d, r.nprob, r.k0, r.nb, r.nbo, r.ival, r.maxc, st, r.cap);
          ++n;
        }
        break;
      case K_LU_BACK: launch_lu_backsub_diag((const LuDesc*)d, r.nprob, r.k0, r.nb, r.maxc, st); ++n; break;
      case K_FROB2: launch_frob2((const Norm1Desc*)d, r.nprob, r.maxc, st); ++n; break;
      case K_NORM1: launch_norm1((const Norm1Desc*)d, r.nprob, r.maxc, st); ++n; break;
      case K_TRACE: launch_trace((const TraceDesc*)d, r.nprob, st); ++n; break;
      case K_EIG: launch_eig((const EigDesc*)d, r.nprob, st); ++n; break;
      case K_CHECK:
        launch_decim_check((double*)r.p[0], (double*)r.p[1], (const double*)r.p[2], (int*)r.p[3],
                           (int*)r.p[4], (int*)r.p[5], r.nprob, r.tol, r.cap, r.count, st);
        ++n;
        break;
      case K_FILL: launch_fill_i32((int*)r.p[0], r.nprob, r.ival, st); ++n; break;
      case K_PACK_A: launch_pack_a((const PackDesc*)d, t, r.nprob, r.tiles, r.ival, st); ++n; break;
      case K_PACK_B: launch_pack_b((const PackDesc*)d, t, r.nprob, r.tiles, r.ival, st); ++n; break;
      case K_TCGEMM: {
        cudaError_t e = launch_tc_gemm((const TcDesc*)d, t, r.nprob, r.tiles, (int*)r.p[0], st);
        if (e != cudaSuccess) return e;
        ++n;
        break;
      }
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
  g_host_calls += n + (long long)std::count_if(recs_.begin(), recs_.end(),
                                                [](const LaunchRec& r) { return r.kind == K_MEMSET; });
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
    graph_sig_ = signature();
  }
  cudaError_t e = cudaGraphLaunch(exec_, st);
  ++g_host_calls;
  if (nlaunch) *nlaunch += graph_kernels_;
  return e;
}

}  // namespace ss
