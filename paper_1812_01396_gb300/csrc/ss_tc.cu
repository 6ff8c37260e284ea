// Complex GEMM on the tcgen05 tensor cores with split-BF16 operands.
//
// The Schur-complement products and the other large contractions of the
// mixed-precision path (Sec. 3C: "two matrix-matrix multiplications" per
// block of Algorithm 1, plus the doubling products) are dense complex GEMMs.
// Each is run as ONE real BF16 GEMM with FP32 accumulation:
//
//   * every FP64 value x is split into BF16 terms x = t0 + t1 (+ t2) with
//     t0 = bf16(x), t1 = bf16(x - t0), t2 = bf16(x - t0 - t1);
//   * a product list picks term pairs (i, j): (0,0),(0,1),(1,0) for the
//     3-product mode, plus (0,2),(2,0),(1,1) for the 6-product mode;
//   * the complex product is the real product [Ar | Ai] x [[Br, Bi], [-Bi, Br]]
//     with the output columns interleaved (re, im), and the term pairs are
//     concatenated along K:  A' = [A_{i0} | A_{i1} | ...],  B' = [B_{j0} | ...].
//
// pack_a / pack_b build A' (m x Kp) and B' (2n x Kp), both K-major BF16, Kp a
// multiple of 64.  tc_gemm multiplies them: one CTA per 128 x 128 tile of
// C' = A' B'^T, TMA loads (128-byte swizzle) into a 4-stage shared-memory
// ring guarded by mbarriers, tcgen05.mma (M = 128, N = 128, K = 16 per
// instruction) issued by one thread into a TMEM accumulator of 128 columns,
// and an epilogue of four warps that reads TMEM with tcgen05.ld and writes
// C = alpha * (C're + i C'im) + beta * Cin in FP64.
//
// Every wait is bounded: after 2 s without progress the kernel records an
// error in *err, stops issuing work, and still frees its TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ss_internal.cuh"
#include "ss_tc.h"
#include "ss_tcutil.cuh"

namespace ss {

namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
constexpr int TC_THREADS = 192;  // warp 0: TMA, warp 1: MMA + TMEM, warps 2-5: epilogue
constexpr uint32_t A_BYTES = BM * BK * 2;
constexpr uint32_t B_BYTES = BN * BK * 2;
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = BN;

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const TcDesc* __restrict__ descs,
                                                                const int* __restrict__ tile_start, int nprob,
                                                                int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the operand ring (required by the swizzle)
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;

  const int pid = find_problem(tile_start, nprob, blockIdx.x);
  const TcDesc& d = descs[pid];
  if (d.active && __ldg(d.active) == 0) return;
  const CUtensorMap* map_a = reinterpret_cast<const CUtensorMap*>(reinterpret_cast<const char*>(descs) + d.ta_off);
  const CUtensorMap* map_b = reinterpret_cast<const CUtensorMap*>(reinterpret_cast<const char*>(descs) + d.tb_off);
  const int tiles_n = (d.n2 + BN - 1) / BN;
  const int t = blockIdx.x - __ldg(tile_start + pid);
  const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BN;
  const int ktiles = d.kp / BK;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) { mbar_init(&full_bar[i], 1); mbar_init(&empty_bar[i], 1); }
    mbar_init(&acc_bar, 1);
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
    for (int kt = 0; kt < ktiles; ++kt) {
      const int st = kt % STAGES;
      const uint32_t ph = (kt / STAGES) & 1;
      if (!mbar_wait(&empty_bar[st], ph ^ 1)) { s_fail = 1; break; }
      unsigned char* sa = smem + st * STAGE_BYTES;
      unsigned char* sb = sa + A_BYTES;
      mbar_expect_tx(&full_bar[st], STAGE_BYTES);
      tma_load_2d(sa, map_a, &full_bar[st], kt * BK, m0);
      tma_load_2d(sb, map_b, &full_bar[st], kt * BK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    bool ok = true;
    for (int kt = 0; kt < ktiles; ++kt) {
      const int st = kt % STAGES;
      const uint32_t ph = (kt / STAGES) & 1;
      if (!mbar_wait(&full_bar[st], ph)) { ok = false; s_fail = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* sa = smem + st * STAGE_BYTES;
      unsigned char* sb = sa + A_BYTES;
      const uint64_t da = smem_desc(sa), db = smem_desc(sb);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) {
        // advance 16 BF16 = 32 bytes along K inside the swizzle atom
        mma_bf16(tmem, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), IDESC, (kt | k) != 0);
      }
      mma_commit(&empty_bar[st]);
    }
    if (ok) mma_commit(&acc_bar);
    else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_bar)) : "memory");
  } else if (warp >= 2) {
    // ---- epilogue: TMEM -> registers -> FP64 complex
    const bool ok = mbar_wait(&acc_bar, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int q = warp & 3;  // TMEM lane quarter this warp may read
    const int row = m0 + q * 32 + lane;
    if (ok && !s_fail) {
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
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
        if (row < d.m) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int col2 = n0 + c * 32 + 2 * e;  // column of C' (re); col2 + 1 is im
            if (col2 < d.n2) {
              const int j = col2 >> 1;
              z64 acc = zmk((double)__uint_as_float(v[2 * e]), (double)__uint_as_float(v[2 * e + 1]));
              z64 out = zmul(d.alpha, acc);
              if (d.cmode == 1) {
                const size_t fi = (size_t)row * d.ldcf + j;
                out = zadd(out, zmul(d.beta, zsub(zmul(d.ce, d.cs[fi]), d.ch[fi])));
              } else if (d.cmode == 2) {
                if (row == j) out = zadd(out, d.beta);
              } else if (d.beta.x != 0.0 || d.beta.y != 0.0) {
                out = zadd(out, zmul(d.beta, d.c[(size_t)row * d.ldc + j]));
              }
              d.c[(size_t)row * d.ldc + j] = out;
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ----------------------------------------------------------------- packing
__device__ __forceinline__ void split3(double x, __nv_bfloat16 (&t)[3]) {
  t[0] = __double2bfloat16(x);
  const double r1 = x - (double)__bfloat162float(t[0]);
  t[1] = __double2bfloat16(r1);
  const double r2 = r1 - (double)__bfloat162float(t[1]);
  t[2] = __double2bfloat16(r2);
}

__device__ __forceinline__ z64 pk_load(const PackDesc& p, int i, int j) {
  // element (i, j) of op(X), X plain or e*S - H
  const size_t idx = p.trans ? (size_t)j * p.ld + i : (size_t)i * p.ld + j;
  z64 v = p.x[idx];
  if (p.s) v = zsub(zmul(p.e, p.s[idx]), v);
  return p.trans ? zconj(v) : v;
}

// A' row r: segments t = 0..nterm-1 of width 2k: [re_term | im_term], then zero pad.
__global__ void pack_a_kernel(const PackDesc* __restrict__ descs, const int* __restrict__ tile_start, int nprob,
                              int mode) {
  const int pid = find_problem(tile_start, nprob, blockIdx.x);
  const PackDesc& p = descs[pid];
  if (p.active && __ldg(p.active) == 0) return;
  const int kk_tiles = (p.kp + 255) / 256;
  const int t = blockIdx.x - __ldg(tile_start + pid);
  const int r = t / kk_tiles;
  const int c = (t % kk_tiles) * 256 + threadIdx.x;  // column of A'
  if (r >= p.rows || c >= p.kp) return;
  const int k = p.k, w2 = 2 * k;
  const int nterm = mode == 2 ? 6 : 3;
  __nv_bfloat16 out = __double2bfloat16(0.0);
  if (c < nterm * w2) {
    const int seg = c / w2, off = c % w2;
    const int kk = off < k ? off : off - k;
    const z64 v = pk_load(p, r, kk);
    __nv_bfloat16 tt[3];
    split3(off < k ? v.x : v.y, tt);
    // A term index per segment: x3: 0,0,1  x6: 0,0,1,0,2,1
    const int aterm = mode == 2 ? (seg == 2 || seg == 5 ? 1 : (seg == 4 ? 2 : 0)) : (seg == 2 ? 1 : 0);
    out = aterm == 0 ? tt[0] : (aterm == 1 ? tt[1] : tt[2]);
  }
  p.out[(size_t)r * p.kp + c] = out;
}

// B' rows 2j (re) and 2j+1 (im) for column j of op(B) (k x n):
//   row 2j   segment: [ Br_term(:, j) | -Bi_term(:, j) ]
//   row 2j+1 segment: [ Bi_term(:, j) |  Br_term(:, j) ]
__global__ void pack_b_kernel(const PackDesc* __restrict__ descs, const int* __restrict__ tile_start, int nprob,
                              int mode) {
  const int pid = find_problem(tile_start, nprob, blockIdx.x);
  const PackDesc& p = descs[pid];
  if (p.active && __ldg(p.active) == 0) return;
  const int kk_tiles = (p.kp + 255) / 256;
  const int t = blockIdx.x - __ldg(tile_start + pid);
  const int r2 = t / kk_tiles;  // row of B' (0 .. 2n-1)
  const int c = (t % kk_tiles) * 256 + threadIdx.x;
  if (r2 >= p.rows || c >= p.kp) return;
  const int k = p.k, w2 = 2 * k;
  const int nterm = mode == 2 ? 6 : 3;
  const int j = r2 >> 1, im_row = r2 & 1;
  __nv_bfloat16 out = __double2bfloat16(0.0);
  if (c < nterm * w2) {
    const int seg = c / w2, off = c % w2;
    const int kk = off < k ? off : off - k;
    const z64 v = pk_load(p, kk, j);
    double x;
    if (!im_row) x = off < k ? v.x : -v.y;
    else x = off < k ? v.y : v.x;
    __nv_bfloat16 tt[3];
    split3(x, tt);
    // B term index per segment: x3: 0,1,0  x6: 0,1,0,2,0,1
    const int bterm = mode == 2 ? (seg == 1 || seg == 5 ? 1 : (seg == 3 ? 2 : 0)) : (seg == 1 ? 1 : 0);
    out = bterm == 0 ? tt[0] : (bterm == 1 ? tt[1] : tt[2]);
  }
  p.out[(size_t)r2 * p.kp + c] = out;
}

}  // namespace

int tc_kp(int k, int mode) {
  const int nterm = mode == 2 ? 6 : 3;
  return ((nterm * 2 * k + BK - 1) / BK) * BK;
}
int tc_tiles(int m, int n2) { return ((m + BM - 1) / BM) * ((n2 + BN - 1) / BN); }
int pack_tiles(int rows, int kp) { return rows * ((kp + 255) / 256); }
size_t tc_smem_bytes() { return (size_t)STAGES * STAGE_BYTES + 1024; }

void launch_pack_a(const PackDesc* d, const int* tile_start, int nprob, int total, int mode, cudaStream_t st) {
  if (nprob <= 0 || total <= 0) return;
  pack_a_kernel<<<total, 256, 0, st>>>(d, tile_start, nprob, mode);
}
void launch_pack_b(const PackDesc* d, const int* tile_start, int nprob, int total, int mode, cudaStream_t st) {
  if (nprob <= 0 || total <= 0) return;
  pack_b_kernel<<<total, 256, 0, st>>>(d, tile_start, nprob, mode);
}
cudaError_t launch_tc_gemm(const TcDesc* d, const int* tile_start, int nprob, int total, int* err, cudaStream_t st) {
  if (nprob <= 0 || total <= 0) return cudaSuccess;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem_bytes());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  tc_gemm_kernel<<<total, TC_THREADS, tc_smem_bytes(), st>>>(d, tile_start, nprob, err);
  return cudaGetLastError();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encode_kmajor_map(CUtensorMap* map, const void* base, int rows, int kp, int box_rows, int ld) {
  if (ld == 0) ld = kp;
  if (ld < kp || (ld * 2) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return cudaErrorInvalidValue;
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tc_box_rows_a() { return BM; }
int tc_box_rows_b() { return BN; }

}  // namespace ss
