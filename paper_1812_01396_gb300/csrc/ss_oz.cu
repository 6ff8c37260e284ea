// FP64-accurate complex GEMM on the tcgen05 tensor cores: digit-sliced
// BF16 operands with exact FP32 accumulation (the Ozaki splitting).
//
// Low-precision products are not usable inside the lead doubling: at
// eta = 1e-10 it amplifies arithmetic error by ~1e6 in band.  So the
// mixed path keeps FP64 accuracy and still runs its products on the tensor
// cores:
//
//   * every row i of op(A) (real-equivalent [Ar | Ai]) gets a power-of-two
//     scale 2^eA[i] >= its largest |entry|, every column j of op(B) a scale
//     2^eB[j] (shared by the re and im rows 2j, 2j+1 of B');
//   * each scaled value r in (-1, 1) is cut into S integer digits of beta bits,
//     r = sum_t d_t 2^{-beta (t+1)}, |d_0| <= 2^beta, |d_t| <= 2^(beta-1) for
//     t > 0 (round to nearest): every digit is an exact BF16 number;
//   * A' = [A_0 | A_1 | ... | A_{S-1}] and B' likewise (each slice w >= 2k
//     wide, zero padded), so the product of digit slices t and u is a plain
//     K-major BF16 GEMM;
//   * slices with the same level d = t + u share the scale 2^{-beta (d+2)};
//     consecutive pairs of one level share one FP32 TMEM accumulator while
//     the sum of their bounds w |d_t| |d_u| stays <= 2^24, so that every
//     partial sum is an integer of at most 24 bits and the FP32 accumulation
//     is EXACT;
//   * each such accumulation ("pass") is drained by the epilogue into an
//     int64 fixed point, scaled by 2^{eA[i] + eB[j] - beta (d+2)} at the end;
//     four TMEM accumulators form a ring so the MMA thread runs ahead of the
//     epilogue.
//
// The digits cover OZ_DIGIT_BITS = 60 bits below each row / column maximum:
// 54 would resolve the largest entries to FP64 precision, the 6 extra keep
// entries up to 64 times smaller than their row maximum at FP64 precision
// too (products pairing a small entry of A with a large one of B otherwise
// lose those bits; on the doubling of the leads this tripled the error of T).
// Levels d <= S - 1 are kept, so the result matches an FP64 GEMM to rounding.
// Persistent CTAs over 128 x 128 tiles of C' = A' B'^T; warp 0 issues TMA,
// warp 1 the MMAs, warps 2-17 drain the accumulators.  Every wait is bounded
// (2 s).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ss_internal.cuh"
#include "ss_tc.h"
#include "ss_tcutil.cuh"

namespace ss {

namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 6, NACC = 4;
constexpr int OZ_DIGIT_BITS = 60;  // bits below the row / column maximum the digits cover
// Tiles of a problem are visited in groups of GM row tiles (column-major
// inside a group), so the CTAs running at the same time share A row panels
// and B column panels and their digit slices stay in L2.
constexpr int GM = 8;
// warp 0: TMA, warp 1: MMA, warps 2-17: epilogue (four warps per TMEM lane
// quadrant, each draining a quarter of the tile's columns: 16 complex
// columns, 32 int64 fixed-point sums per thread).  The drain of every pass is
// the bound of the small-k products; sixteen draining warps (rather than
// eight with twice the sums each) measured 9 % faster on the LU's k = 64
// updates.
constexpr int EPI_WARPS = 16;
constexpr int EPI_COLS = BN / (EPI_WARPS / 4);  // real columns per epilogue thread
constexpr int OZ_THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t A_BYTES = BM * BK * 2;
constexpr uint32_t B_BYTES = BN * BK * 2;
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = NACC * BN;  // NACC accumulators of BN columns (512 = all of TMEM)
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ double pow2(int e) {
  // 2^e: built from the exponent bits in the normal range, ldexp outside it
  if (e > -1020 && e < 1020) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

// Exponent e with max < 2^e from the IEEE bits of a non-negative maximum
// (0 for an all-zero vector; subnormal maxima use the smallest normal scale).
__device__ __forceinline__ int exp_of(unsigned long long mx) {
  const int ex = (int)(mx >> 52);
  return mx == 0 ? 0 : (ex == 0 ? -1021 : ex - 1022);
}

// Persistent: CTA c processes tiles c, c + gridDim.x, ...  The three roles
// walk the same tile sequence; the stage ring (producer -> MMA) and the
// accumulator ring (MMA -> epilogue) continue across tiles, so the epilogue
// of one tile overlaps the MMAs of the next, and TMEM is allocated once.
__device__ __forceinline__ bool oz_tile(const OzDesc* __restrict__ descs, const int* __restrict__ tile_start,
                                        int nprob, int tile, int& pid, int& m0, int& n0) {
  pid = find_problem(tile_start, nprob, tile);
  const OzDesc& d = descs[pid];
  if (d.active && __ldg(d.active) == 0) return false;
  const int tiles_n = (d.n2 + BN - 1) / BN, tiles_m = (d.m + BM - 1) / BM;
  const int t = tile - __ldg(tile_start + pid);
  const int group = t / (GM * tiles_n), first = group * GM;
  const int gm = min(GM, tiles_m - first), r = t - group * GM * tiles_n;
  m0 = (first + r % gm) * BM;
  n0 = (r / gm) * BN;
  if (d.lower && (n0 >> 1) >= m0 + BM) return false;  // tile entirely above the diagonal
  return true;
}

__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(const OzDesc* __restrict__ descs,
                                                                const int* __restrict__ tile_start, int nprob,
                                                                int total_tiles, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[NACC];
  __shared__ __align__(8) uint64_t acce_bar[NACC];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_fail;
  __shared__ double colscale[BN / 2];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) { mbar_init(&full_bar[i], 1); mbar_init(&empty_bar[i], 1); }
    for (int i = 0; i < NACC; ++i) { mbar_init(&accf_bar[i], 1); mbar_init(&acce_bar[i], 32 * EPI_WARPS); }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    int kt = 0;
    for (int tile = blockIdx.x; tile < total_tiles && !s_fail; tile += gridDim.x) {
      int pid, m0, n0;
      if (!oz_tile(descs, tile_start, nprob, tile, pid, m0, n0)) continue;
      const OzDesc& d = descs[pid];
      const CUtensorMap* map_a = reinterpret_cast<const CUtensorMap*>(reinterpret_cast<const char*>(descs) + d.ta_off);
      const CUtensorMap* map_b = reinterpret_cast<const CUtensorMap*>(reinterpret_cast<const char*>(descs) + d.tb_off);
      const int wt = d.w / BK;
      for (int p = 0; p < d.npass && !s_fail; ++p) {
        const int lev = d.pd[p], t0 = d.pt0[p], np = d.pnp[p];
        for (int q = 0; q < np && !s_fail; ++q) {
          const int ta = t0 + q, tb = lev - ta;
          for (int kk = 0; kk < wt; ++kk, ++kt) {
            const int st = kt % STAGES;
            const uint32_t ph = (kt / STAGES) & 1;
            if (!mbar_wait(&empty_bar[st], ph ^ 1)) { s_fail = 1; break; }
            unsigned char* sa = smem + st * STAGE_BYTES;
            unsigned char* sb = sa + A_BYTES;
            mbar_expect_tx(&full_bar[st], STAGE_BYTES);
            tma_load_2d(sa, map_a, &full_bar[st], ta * d.w + kk * BK, m0);
            tma_load_2d(sb, map_b, &full_bar[st], tb * d.w + kk * BK, n0);
          }
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: one accumulator of the ring per pass
    int kt = 0, pg = 0;
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
      int pid, m0, n0;
      if (!oz_tile(descs, tile_start, nprob, tile, pid, m0, n0)) continue;
      const OzDesc& d = descs[pid];
      const int wt = d.w / BK;
      for (int p = 0; p < d.npass; ++p, ++pg) {
        const int acc = pg % NACC, use = pg / NACC;
        bool ok = !s_fail && mbar_wait(&acce_bar[acc], (use & 1) ^ 1);
        if (!ok) s_fail = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int nk = d.pnp[p] * wt;
        for (int i = 0; i < nk && ok; ++i, ++kt) {
          const int st = kt % STAGES;
          const uint32_t ph = (kt / STAGES) & 1;
          if (!mbar_wait(&full_bar[st], ph)) { ok = false; s_fail = 1; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          unsigned char* sa = smem + st * STAGE_BYTES;
          unsigned char* sb = sa + A_BYTES;
          const uint64_t da = smem_desc(sa), db = smem_desc(sb);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)
            mma_bf16(tmem + acc * BN, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), IDESC, (i | k) != 0);
          mma_commit(&empty_bar[st]);
        }
        if (ok) mma_commit(&accf_bar[acc]);
        else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&accf_bar[acc])) : "memory");
      }
    }
  } else if (warp >= 2) {
    // ---- epilogue: drain every pass of every tile into int64 fixed point
    // Every pass sum is an exact integer below 2^24.  They are added in
    // int64 fixed point with FIX = 37 fractional bits of the level-0 unit
    // (|total| < 2^24 * 1.1 * 2^37 < 2^62): levels with beta*d <= 37 are
    // exact, deeper ones round by at most half a unit of 2^-37, so FP64
    // arithmetic is needed only once per output element.
    const int q4 = warp & 3;             // TMEM lanes 32 q4 .. 32 q4 + 31
    const int part = (warp - 2) >> 2;    // real columns EPI_COLS part .. of the tile
    static_assert(EPI_COLS % 8 == 0, "8-column TMEM loads");
    int pg = 0;
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
      int pid, m0, n0;
      if (!oz_tile(descs, tile_start, nprob, tile, pid, m0, n0)) continue;
      const OzDesc& d = descs[pid];
      const int row = m0 + q4 * 32 + lane;
      if (threadIdx.x - 64 < BN / 2) {
        const int j = (n0 >> 1) + (threadIdx.x - 64);
        colscale[threadIdx.x - 64] = (2 * j < d.n2) ? pow2(exp_of(d.mB[j])) : 0.0;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * EPI_WARPS) : "memory");  // epilogue warps only
      long long re[EPI_COLS / 2], im[EPI_COLS / 2];
#pragma unroll
      for (int e = 0; e < EPI_COLS / 2; ++e) { re[e] = 0; im[e] = 0; }
      bool ok = true;
      for (int p = 0; p < d.npass; ++p, ++pg) {
        const int acc = pg % NACC, use = pg / NACC;
        if (ok && !s_fail && !mbar_wait(&accf_bar[acc], use & 1)) { ok = false; s_fail = 1; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int sh = 37 - d.beta_bits * d.pd[p];  // shift of this level into the fixed point
        if (ok && !s_fail) {
#pragma unroll
          for (int sub = 0; sub < EPI_COLS / 8; ++sub) {
            uint32_t v[8];
            const uint32_t taddr =
                tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(acc * BN + part * EPI_COLS + sub * 8);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (sh >= 0) {
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                re[sub * 4 + e] += (long long)__float2int_rn(__uint_as_float(v[2 * e])) << sh;
                im[sub * 4 + e] += (long long)__float2int_rn(__uint_as_float(v[2 * e + 1])) << sh;
              }
            } else {
              const int rs = -sh;
              const long long rnd = 1ll << (rs - 1);
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                re[sub * 4 + e] += ((long long)__float2int_rn(__uint_as_float(v[2 * e])) + rnd) >> rs;
                im[sub * 4 + e] += ((long long)__float2int_rn(__uint_as_float(v[2 * e + 1])) + rnd) >> rs;
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[acc])) : "memory");
      }
      if (ok && !s_fail && row < d.m) {
        // value = fixed / 2^37 * 2^{-2 beta} * 2^{eA[row]} * 2^{eB[j]}
        const double rs_row = pow2(exp_of(d.mA[row]) - 37 - 2 * d.beta_bits);
        const bool unit_alpha = d.alpha.y == 0.0 && (d.alpha.x == 1.0 || d.alpha.x == -1.0);
#pragma unroll
        for (int e = 0; e < EPI_COLS / 2; ++e) {
          const int j = (n0 >> 1) + part * (EPI_COLS / 2) + e;
          if (2 * j < d.n2) {
            const double sc = rs_row * colscale[part * (EPI_COLS / 2) + e];
            z64 out = zmk((double)re[e] * sc, (double)im[e] * sc);
            if (unit_alpha) { if (d.alpha.x < 0.0) { out.x = -out.x; out.y = -out.y; } }
            else out = zmul(d.alpha, out);
            if (d.cmode == 1) {
              const size_t fi = (size_t)row * d.ldcf + j;
              out = zadd(out, zmul(d.beta, zsub(zmul(d.ce, d.cs[fi]), d.ch[fi])));
            } else if (d.cmode == 2) {
              if (row == j) out = zadd(out, d.beta);
            } else if (d.beta.y == 0.0 && d.beta.x != 0.0) {  // real beta: two FMAs
              const z64 cv = d.c[(size_t)row * d.ldc + j];
              out = zmk(fma(d.beta.x, cv.x, out.x), fma(d.beta.x, cv.y, out.y));
            } else if (d.beta.x != 0.0 || d.beta.y != 0.0) {
              out = zadd(out, zmul(d.beta, d.c[(size_t)row * d.ldc + j]));
            }
            d.c[(size_t)row * d.ldc + j] = out;
          }
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * EPI_WARPS) : "memory");  // colscale is rewritten next tile
    }
  }
  __syncthreads();
  if (s_fail && threadIdx.x == 0 && err) atomicExch(err, 1);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// --------------------------------------------------------------- scaling
__device__ __forceinline__ z64 oz_load(const OzPackDesc& p, int i, int j) {
  const size_t idx = p.trans ? (size_t)j * p.ld + i : (size_t)i * p.ld + j;
  z64 v = p.x[idx];
  if (p.s) {  // e S - H; real e (the device at real E) needs two FMAs, not a complex product
    const z64 sv = p.s[idx];
    v = p.e.y == 0.0 ? zmk(fma(p.e.x, sv.x, -v.x), fma(p.e.x, sv.y, -v.y)) : zsub(zmul(p.e, sv), v);
  }
  return p.trans ? zconj(v) : v;
}

// The (vector, inner) index of op(X): vector = row of op(A) (role 0) or
// column of op(B) (role 1).  `contig_inner` tells which index runs along
// memory, so tiles are loaded with consecutive threads on consecutive
// addresses whatever the operand's orientation.
__device__ __forceinline__ bool contig_inner(const OzPackDesc& p) {
  return (p.role == 0 && !p.trans) || (p.role == 1 && p.trans);
}
__device__ __forceinline__ z64 oz_elem(const OzPackDesc& p, int v, int kk) {
  return p.role == 0 ? oz_load(p, v, kk) : oz_load(p, kk, v);
}

// Per-vector maximum of max(|re|, |im|) over a 32 x 32 tile, merged with
// an integer atomicMax on the IEEE bits (monotone for non-negative values).
__global__ void __launch_bounds__(256) oz_scale_kernel(const OzPackDesc* __restrict__ descs,
                                                       const int* __restrict__ tile_start, int nprob) {
  const int pid = find_problem(tile_start, nprob, blockIdx.x);
  const OzPackDesc& p = descs[pid];
  if (p.active && __ldg(p.active) == 0) return;
  const int nvec = p.role == 0 ? p.rows : p.rows / 2;
  const int kt = (p.k + 31) / 32;
  const int t = blockIdx.x - __ldg(tile_start + pid);
  const int v0 = (t / kt) * 32, k0 = (t % kt) * 32;
  __shared__ unsigned long long tile[32][33];
  const bool ci = contig_inner(p);
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int a = e / 32, b = e % 32;  // b runs along memory
    const int v = v0 + (ci ? a : b), kk = k0 + (ci ? b : a);
    unsigned long long m = 0;
    if (v < nvec && kk < p.k) {
      const z64 z = oz_elem(p, v, kk);
      const unsigned long long x = (unsigned long long)__double_as_longlong(z.x) & 0x7FFFFFFFFFFFFFFFull;
      const unsigned long long y = (unsigned long long)__double_as_longlong(z.y) & 0x7FFFFFFFFFFFFFFFull;
      m = x > y ? x : y;
    }
    tile[ci ? a : b][ci ? b : a] = m;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int v = v0 + threadIdx.x;
    unsigned long long m = 0;
    for (int j = 0; j < 32; ++j) m = tile[threadIdx.x][j] > m ? tile[threadIdx.x][j] : m;
    if (v < nvec && m) atomicMax(p.maxb + v, m);
  }
}

// Signed 62-bit fixed point R = x 2^{62-e} of |x| < 2^e from the IEEE bits
// (zero and subnormals, far below any row scale here, give zero).
__device__ __forceinline__ long long fixed62(double x, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long R = 0;
  if (ex != 0) {
    const long long m = (long long)((bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
    const int shift = ex - 1013 - e;  // x 2^{62-e} = m 2^{ex-1075+62-e}
    if (shift >= 0) R = m << shift;   // shift <= 9 because |x| < 2^e
    else if (shift > -64) R = (m + (1ll << (-shift - 1))) >> (-shift);
    if (bits >> 63) R = -R;
  }
  return R;
}

// Digit t of R is the round-to-nearest quotient by 2^{62 - beta (t+1)}, then
// removed from R (a digit past the 62 fixed-point bits, beta S > 62, is the
// remainder scaled up, exactly); |digit| <= 2^beta is an exact BF16 number.  Two values
// (adjacent columns) at a time, stored as one bfloat16 pair per slice.
template <int S>
__device__ __forceinline__ void write_digits2(__nv_bfloat16* row, int w, int off, int beta, double x0, double x1,
                                              int e) {
  long long R0 = fixed62(x0, e), R1 = fixed62(x1, e);
#pragma unroll 3
  for (int t = 0; t < S; ++t) {
    const int sh = 62 - beta * (t + 1);
    long long q0, q1;
    if (sh > 0) {
      const long long h = 1ll << (sh - 1);
      q0 = (R0 + h) >> sh;
      q1 = (R1 + h) >> sh;
      R0 -= q0 << sh;
      R1 -= q1 << sh;
    } else {  // past the 62 fixed-point bits: the remainder itself, exactly
      q0 = R0 << -sh;
      q1 = R1 << -sh;
      R0 = R1 = 0;
    }
    *reinterpret_cast<__nv_bfloat162*>(row + (size_t)t * w + off) =
        __floats2bfloat162_rn((float)(int)q0, (float)(int)q1);
  }
}

// The same digits written to two places: row d0 at off0 (negated when neg0:
// the digits of -x are exactly the negated digits of x) and row d1 at off1.
// B' holds every value of op(B) twice ([Br | -Bi] and [Bi | Br]), so its
// digits are extracted once.
template <int S>
__device__ __forceinline__ void write_digits2x(__nv_bfloat16* d0, int off0, bool neg0, __nv_bfloat16* d1, int off1,
                                               int w, int beta, double x0, double x1, int e) {
  long long R0 = fixed62(x0, e), R1 = fixed62(x1, e);
#pragma unroll 3
  for (int t = 0; t < S; ++t) {
    const int sh = 62 - beta * (t + 1);
    long long q0, q1;
    if (sh > 0) {
      const long long h = 1ll << (sh - 1);
      q0 = (R0 + h) >> sh;
      q1 = (R1 + h) >> sh;
      R0 -= q0 << sh;
      R1 -= q1 << sh;
    } else {
      q0 = R0 << -sh;
      q1 = R1 << -sh;
      R0 = R1 = 0;
    }
    const float f0 = (float)(int)q0, f1 = (float)(int)q1;
    const __nv_bfloat162 v = __floats2bfloat162_rn(f0, f1);
    *reinterpret_cast<__nv_bfloat162*>(d0 + (size_t)t * w + off0) = neg0 ? __floats2bfloat162_rn(-f0, -f1) : v;
    *reinterpret_cast<__nv_bfloat162*>(d1 + (size_t)t * w + off1) = v;
  }
}

template <int S>
__device__ __forceinline__ void write_digits1x(__nv_bfloat16* d0, int off0, bool neg0, __nv_bfloat16* d1, int off1,
                                               int w, int beta, double x, int e) {
  long long R = fixed62(x, e);
#pragma unroll 3
  for (int t = 0; t < S; ++t) {
    const int sh = 62 - beta * (t + 1);
    long long q;
    if (sh > 0) {
      q = (R + (1ll << (sh - 1))) >> sh;
      R -= q << sh;
    } else {
      q = R << -sh;
      R = 0;
    }
    const float f = (float)(int)q;
    d0[(size_t)t * w + off0] = __float2bfloat16_rn(neg0 ? -f : f);
    d1[(size_t)t * w + off1] = __float2bfloat16_rn(f);
  }
}

template <int S>
__device__ __forceinline__ void write_digits1(__nv_bfloat16* row, int w, int off, int beta, double x, int e) {
  long long R = fixed62(x, e);
#pragma unroll 3
  for (int t = 0; t < S; ++t) {
    const int sh = 62 - beta * (t + 1);
    long long q;
    if (sh > 0) {
      q = (R + (1ll << (sh - 1))) >> sh;
      R -= q << sh;
    } else {  // past the 62 fixed-point bits: the remainder itself, exactly
      q = R << -sh;
      R = 0;
    }
    row[(size_t)t * w + off] = __float2bfloat16_rn((float)(int)q);
  }
}

// Digit slices of a 32 x 32 tile (coalesced loads into shared memory, then
// rows of the packed matrix written along the inner index, two columns per
// thread when k is even), or, for the tiles past the data, the zero padding
// of every slice.
template <int S>
__device__ __forceinline__ void pack_tile(const OzPackDesc& p, int t, z64 (&tile)[32][33], int (&ex)[32]) {
  const int nvec = p.role == 0 ? p.rows : p.rows / 2;
  const int k = p.k;
  const int kt = (k + 31) / 32, pt = (p.w - 2 * k + 31) / 32;
  const int v0 = (t / (kt + pt)) * 32, ti = t % (kt + pt);
  const int nrow_per_vec = p.role == 0 ? 1 : 2;
  const size_t rowlen = (size_t)S * p.w;
  if (ti >= kt) {  // zero padding columns [2k + 32 (ti - kt), ...)
    const int c0 = 2 * k + 32 * (ti - kt);
    for (int e = threadIdx.x; e < 32 * 32 * nrow_per_vec; e += 256) {
      const int c = c0 + (e % 32), vr = e / 32;
      const int v = v0 + vr / nrow_per_vec;
      if (v >= nvec || c >= p.w) continue;
      const int row = p.role == 0 ? v : 2 * v + (vr % 2);
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) p.out[(size_t)row * rowlen + (size_t)s2 * p.w + c] = __double2bfloat16(0.0);
    }
    return;
  }
  const int k0 = ti * 32;
  const bool ci = contig_inner(p);
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int a = e / 32, b = e % 32;
    const int vv = ci ? a : b, kk = ci ? b : a;
    const int v = v0 + vv, kg = k0 + kk;
    tile[vv][kk] = (v < nvec && kg < k) ? oz_elem(p, v, kg) : zmk(0.0, 0.0);
  }
  if (threadIdx.x < 32) ex[threadIdx.x] = v0 + threadIdx.x < nvec ? exp_of(p.maxb[v0 + threadIdx.x]) : 0;
  __syncthreads();
  const int beta = p.beta_bits;
  if ((k & 1) == 0) {
    for (int e = threadIdx.x; e < 512; e += 256) {
      const int vv = e / 16, kk = 2 * (e % 16);
      const int v = v0 + vv, kg = k0 + kk;
      if (v >= nvec || kg >= k) continue;  // k even: kg + 1 < k as well
      const z64 z0 = tile[vv][kk], z1 = tile[vv][kk + 1];
      if (p.role == 0) {  // A' row v = [Ar | Ai]
        __nv_bfloat16* row = p.out + (size_t)v * rowlen;
        write_digits2<S>(row, p.w, kg, beta, z0.x, z1.x, ex[vv]);
        write_digits2<S>(row, p.w, k + kg, beta, z0.y, z1.y, ex[vv]);
      } else {  // B' rows 2v = [Br | -Bi], 2v+1 = [Bi | Br]
        __nv_bfloat16* r0 = p.out + (size_t)(2 * v) * rowlen;
        __nv_bfloat16* r1 = r0 + rowlen;
        write_digits2x<S>(r0, kg, false, r1, k + kg, p.w, beta, z0.x, z1.x, ex[vv]);  // Br
        write_digits2x<S>(r0, k + kg, true, r1, kg, p.w, beta, z0.y, z1.y, ex[vv]);  // -Bi, Bi
      }
    }
    return;
  }
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int vv = e / 32, kk = e % 32;
    const int v = v0 + vv, kg = k0 + kk;
    if (v >= nvec || kg >= k) continue;
    const z64 z = tile[vv][kk];
    if (p.role == 0) {
      __nv_bfloat16* row = p.out + (size_t)v * rowlen;
      write_digits1<S>(row, p.w, kg, beta, z.x, ex[vv]);
      write_digits1<S>(row, p.w, k + kg, beta, z.y, ex[vv]);
    } else {
      __nv_bfloat16* r0 = p.out + (size_t)(2 * v) * rowlen;
      __nv_bfloat16* r1 = r0 + rowlen;
      write_digits1x<S>(r0, kg, false, r1, k + kg, p.w, beta, z.x, ex[vv]);  // Br
      write_digits1x<S>(r0, k + kg, true, r1, kg, p.w, beta, z.y, ex[vv]);  // -Bi, Bi
    }
  }
}

__global__ void __launch_bounds__(256, 3) oz_pack_kernel(const OzPackDesc* __restrict__ descs,
                                                      const int* __restrict__ tile_start, int nprob) {
  const int pid = find_problem(tile_start, nprob, blockIdx.x);
  const OzPackDesc& p = descs[pid];
  if (p.active && __ldg(p.active) == 0) return;
  __shared__ z64 tile[32][33];
  __shared__ int ex[32];
  const int t = blockIdx.x - __ldg(tile_start + pid);
  switch (p.S) {  // the slice counts oz_plan produces (beta 8 .. 3)
    case 8: pack_tile<8>(p, t, tile, ex); break;
    case 9: pack_tile<9>(p, t, tile, ex); break;
    case 10: pack_tile<10>(p, t, tile, ex); break;
    case 12: pack_tile<12>(p, t, tile, ex); break;
    case 15: pack_tile<15>(p, t, tile, ex); break;
    case 20: pack_tile<20>(p, t, tile, ex); break;
    default: break;
  }
}

}  // namespace

size_t oz_smem_bytes() { return (size_t)STAGES * STAGE_BYTES + 1024; }
int oz_tiles(int m, int n2) { return ((m + BM - 1) / BM) * ((n2 + BN - 1) / BN); }
int oz_scale_tiles(const OzPackDesc& d) {
  const int nvec = d.role == 0 ? d.rows : d.rows / 2;
  return ((nvec + 31) / 32) * ((d.k + 31) / 32);
}
int oz_pack_tiles(const OzPackDesc& d) {
  const int nvec = d.role == 0 ? d.rows : d.rows / 2;
  return ((nvec + 31) / 32) * ((d.k + 31) / 32 + (d.w - 2 * d.k + 31) / 32);
}
int oz_box_rows_a() { return BM; }
int oz_box_rows_b() { return BN; }

// Choose beta (bits per digit) for slices of width w: S = ceil(60 / beta)
// slices.  Digit bounds: the leading digit of a value is at most 2^beta in
// magnitude, every later digit at most 2^(beta-1) (round to nearest leaves a
// remainder of at most half a unit), so a digit pair (t, u) contributes at
// most w * 2^(2 beta - [t>0] - [u>0]) to a pass.  The pairs of one level are
// packed into passes greedily while that sum stays <= 2^24 (every partial sum
// then an integer an FP32 accumulator holds exactly).  Cost = tensor K-tiles
// (pairs * w / 64) plus about four K-tiles per pass drained by the epilogue;
// the cheapest beta with at most OZ_MAXPASS passes wins.  beta <= 8 keeps every
// digit (|d| <= 256) an exact BF16 number.
namespace {
int oz_passes(int w, int beta, int S, OzShape* out) {
  const double cap = 16777216.0;
  int n = 0;
  for (int lev = 0; lev < S; ++lev) {
    int t0 = 0;
    double acc = 0.0;
    for (int t = 0; t <= lev; ++t) {
      const int e = 2 * beta - (t > 0) - (lev - t > 0);
      const double b = (double)w * (double)(1ll << e);
      if (b > cap) return OZ_MAXPASS + 1;  // one pair alone is not exact
      if (acc + b > cap) {                 // close the pass [t0, t)
        if (out && n < OZ_MAXPASS) { out->pd[n] = (unsigned char)lev; out->pt0[n] = (unsigned char)t0; out->pnp[n] = (unsigned char)(t - t0); }
        ++n;
        t0 = t;
        acc = 0.0;
      }
      acc += b;
    }
    if (out && n < OZ_MAXPASS) { out->pd[n] = (unsigned char)lev; out->pt0[n] = (unsigned char)t0; out->pnp[n] = (unsigned char)(lev + 1 - t0); }
    ++n;
  }
  return n;
}
}  // namespace

void oz_plan(int k, OzShape* sh) {
  const int w = ((2 * k + BK - 1) / BK) * BK;
  int best_beta = -1, best_S = 0;
  double best_cost = 0.0;
  for (int beta = 8; beta >= 3; --beta) {
    const int S = (OZ_DIGIT_BITS + beta - 1) / beta;  // 8, 9, 10, 12, 15, 20: the packing kernel's instances
    const int npass = oz_passes(w, beta, S, nullptr);
    if (npass > OZ_MAXPASS) continue;
    const double cost = (double)S * (S + 1) / 2 * (w / BK) + 4.0 * npass;
    if (best_beta < 0 || cost < best_cost) { best_beta = beta; best_S = S; best_cost = cost; }
  }
  sh->w = w;
  sh->npass = 0;
  if (best_beta < 0) {  // no exact split for this width: caller must not use the kernel
    sh->beta = 0;
    sh->S = 0;
    sh->npass = OZ_MAXPASS + 1;
    return;
  }
  sh->beta = best_beta;
  sh->S = best_S;
  sh->npass = oz_passes(w, best_beta, best_S, sh);
}

void launch_oz_scale(const OzPackDesc* d, const int* tile_start, int nprob, int total, cudaStream_t st) {
  if (nprob <= 0 || total <= 0) return;
  oz_scale_kernel<<<total, 256, 0, st>>>(d, tile_start, nprob);
}
void launch_oz_pack(const OzPackDesc* d, const int* tile_start, int nprob, int total, cudaStream_t st) {
  if (nprob <= 0 || total <= 0) return;
  oz_pack_kernel<<<total, 256, 0, st>>>(d, tile_start, nprob);
}
cudaError_t launch_oz_gemm(const OzDesc* d, const int* tile_start, int nprob, int total, int* err, cudaStream_t st) {
  if (nprob <= 0 || total <= 0) return cudaSuccess;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)oz_smem_bytes());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 148;
  }
  const int grid = total < nsm ? total : nsm;  // persistent: one CTA per SM
  oz_gemm_kernel<<<grid, OZ_THREADS, oz_smem_bytes(), st>>>(d, tile_start, nprob, total, err);
  return cudaGetLastError();
}

}  // namespace ss
