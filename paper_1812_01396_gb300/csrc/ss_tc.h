// Tensor-core (tcgen05) complex GEMM: descriptors and launchers.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ss_internal.cuh"

namespace ss {

// Packing of one complex operand into split-BF16 real form (see ss_tc.cu).
// For A: rows = m, element (i, kk) of op(X) for i < m, kk < k.
// For B: rows = 2n, element (kk, j) of op(X) for kk < k, j < n.
struct PackDesc {
  const z64* x;     // plain matrix, or H of a formed operand
  const z64* s;     // S of a formed operand (e*S - H), else null
  z64 e;
  int ld, trans;
  int rows, k, kp;  // packed matrix is rows x kp, row-major BF16
  __nv_bfloat16* out;
  const int* active;
};

// One real GEMM C' = A' B'^T (m x n2, n2 = 2n) with the complex epilogue
// C = alpha (C're + i C'im) + beta Cin (cmode as in GemmDesc).
struct TcDesc {
  long long ta_off;  // byte offsets of the two 64-byte aligned tensor maps,
  long long tb_off;  // relative to the start of the TcDesc array
  int m, n2, kp;
  int kc;  // complex inner dimension (for the algorithmic flop count)
  z64* c;
  int ldc;
  int cmode;
  z64 alpha, beta;
  const z64* cs;
  const z64* ch;
  z64 ce;
  int ldcf;
  const int* active;
};

// ---- FP64-accurate digit-sliced GEMM (ss_oz.cu)
constexpr int OZ_MAXPASS = 32;

// Slicing of one inner dimension k: slice width w (>= 2k, multiple of 64),
// beta bits per digit, S slices, and the passes (level d, first slice t0,
// number of pairs np) whose FP32 sums are exact.
struct OzShape {
  int w, beta, S, npass;
  unsigned char pd[OZ_MAXPASS], pt0[OZ_MAXPASS], pnp[OZ_MAXPASS];
};
void oz_plan(int k, OzShape* sh);

// One operand to scale and slice.  role 0: A (rows = m, vectors = rows of
// op(X)); role 1: B (rows = 2n, vectors = columns of op(X)).
struct OzPackDesc {
  const z64* x;
  const z64* s;
  z64 e;
  int ld, trans, role;
  int rows, k, w, S, beta_bits;
  unsigned long long* maxb;  // per-vector max |entry| as IEEE bits (zeroed before the scale pass)
  __nv_bfloat16* out;   // rows x (S * w) row-major
  const int* active;
};

struct OzDesc {
  long long ta_off, tb_off;  // tensor maps, relative to the start of the OzDesc array
  int m, n2, w, kc, beta_bits, npass;
  unsigned char pd[OZ_MAXPASS], pt0[OZ_MAXPASS], pnp[OZ_MAXPASS];
  const unsigned long long* mA;  // row maxima of op(A) (IEEE bits)
  const unsigned long long* mB;  // column maxima of op(B)
  z64* c;
  int ldc;
  int cmode;
  z64 alpha, beta;
  const z64* cs;
  const z64* ch;
  z64 ce;
  int ldcf;
  const int* active;
  int lower;  // skip tiles entirely above the diagonal (complex indices)
};

size_t oz_smem_bytes();
int oz_tiles(int m, int n2);
int oz_box_rows_a();
int oz_box_rows_b();
// tiles of 32 vectors x 32 inner indices; pack also covers the zero padding
int oz_scale_tiles(const OzPackDesc& d);
int oz_pack_tiles(const OzPackDesc& d);
void launch_oz_scale(const OzPackDesc* d, const int* tile_start, int nprob, int total, cudaStream_t st);
void launch_oz_pack(const OzPackDesc* d, const int* tile_start, int nprob, int total, cudaStream_t st);
cudaError_t launch_oz_gemm(const OzDesc* d, const int* tile_start, int nprob, int total, int* err,
                           cudaStream_t st);

int tc_kp(int k, int mode);           // padded packed K for mode 1 (3 products) / 2 (6 products)
int tc_tiles(int m, int n2);
int pack_tiles(int rows, int kp);
size_t tc_smem_bytes();
int tc_box_rows_a();
int tc_box_rows_b();
// Tensor map of a K-major BF16 matrix (rows x kp, row stride ld elements, ld = kp when 0;
// ld * 2 must be a multiple of 16 bytes), box 64 x box_rows, 128-byte swizzle, zero fill
// outside the matrix.
cudaError_t encode_kmajor_map(CUtensorMap* map, const void* base, int rows, int kp, int box_rows, int ld = 0);

void launch_pack_a(const PackDesc* d, const int* tile_start, int nprob, int total, int mode, cudaStream_t st);
void launch_pack_b(const PackDesc* d, const int* tile_start, int nprob, int total, int mode, cudaStream_t st);
cudaError_t launch_tc_gemm(const TcDesc* d, const int* tile_start, int nprob, int total, int* err,
                           cudaStream_t st);

}  // namespace ss
