// Internal declarations of the SplitSolve CUDA library: batched-problem
// descriptors, complex helpers and kernel launchers.
//
// Every heavy kernel works on a *group* of independent problems (one per
// (E,k) point, sweep direction or lead) described by an array of descriptors in
// device memory, so that points with different block sizes run in one launch.
// A descriptor may carry an `active` flag pointer: a problem whose flag is 0
// is skipped (converged doubling, finished refinement).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace ss {

typedef double2 z64;

__host__ __device__ __forceinline__ z64 zmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ z64 zadd(z64 a, z64 b) { return zmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ z64 zsub(z64 a, z64 b) { return zmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ z64 zmul(z64 a, z64 b) {
  return zmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ z64 zconj(z64 a) { return zmk(a.x, -a.y); }
// acc += a * b with four fused multiply-adds
__device__ __forceinline__ void zfma(z64& acc, z64 a, z64 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// 1 / a, scaled to avoid overflow of |a|^2
__device__ __forceinline__ z64 zinv(z64 a) {
  double s = fmax(fabs(a.x), fabs(a.y));
  if (s == 0.0) return zmk(0.0, 0.0);
  double ar = a.x / s, ai = a.y / s;
  double d = ar * ar + ai * ai;
  return zmk(ar / (d * s), -ai / (d * s));
}

// ---------------------------------------------------------------- operands
// A matrix operand: plain (p) or formed on the fly as e*S - H (s != nullptr,
// p = H), optionally conjugate-transposed.  ld is the row stride in elements.
struct Operand {
  const z64* p;
  const z64* s;
  z64 e;
  int ld;
  int trans;  // 0: op(X) = X, 1: op(X) = X^H
};

// C = alpha * op(A) op(B) + beta * Cin, Cin = C (cmode 0), e*S - H (cmode 1,
// from cs/ch with ld ldcf) or the identity (cmode 2).
struct GemmDesc {
  int m, n, k;
  Operand a, b;
  z64* c;
  int ldc;
  int cmode;
  z64 alpha, beta;
  const z64* cs;
  const z64* ch;
  z64 ce;
  int ldcf;
  const int* active;
  int lower;  // 1: only the lower triangle of C (m = n) is needed; tiles above the diagonal are skipped
};

// Elementwise out = ax*op(X) + ay*op(Y) + az*op(Z) + gamma*I over rows x cols.
// Operands may be null (zero).  In-place use needs trans = 0 on aliases.
struct FormDesc {
  z64* out;
  int ldo, rows, cols;
  const z64* x; int ldx; int tx; z64 ax;
  const z64* y; int ldy; int ty; z64 ay;
  const z64* z; int ldz; int tz; z64 az;
  z64 gamma;
  const int* active;
  const z64* v; int ldv; z64 av;  // fourth term (not transposed)
  // norm mode (nrm != nullptr): nothing is written; *nrm += nw * sum |value|^2
  double* nrm; double nw;
};

// Blocked LU with partial pivoting of the leading s x s block of the
// row-major s x ncols matrix w, with columns s..ncols-1 as right-hand sides.
struct LuDesc {
  z64* w;
  int ldw;
  int s;
  int ncols;
  int* ipiv;     // s entries, absolute row index swapped with row j at step j
  int* info;     // 0, or 1 + first column with a zero / non-finite pivot
  const int* active;
};

// Dense complex eigenproblem K y = lambda y of size m <= 512 (ss_eig.cu):
// h holds K on entry and its Schur form T on exit, z receives the unitary
// Z with K = Z T Z^H, x the eigenvectors of T (column j for lam[j]; the
// eigenvectors of K are Z x), all m x m with leading dimension ld.
struct EigDesc {
  z64* h;
  z64* z;
  z64* x;
  z64* lam;
  int m, ld;
  int* info;  // 1 if the QR iteration hit its cap
};
void launch_eig(const EigDesc* d, int nprob, cudaStream_t st);

// Norm / reduction descriptors
struct Norm1Desc {
  const z64* a; int lda; int rows, cols;
  double* out;  // max column sum of moduli |a_ij|; must hold 0.0 before the launch
  const int* active;
};

struct TraceDesc {  // out = sum_{a,b} A[a,b] * B[b,a]; b == nullptr: out = sum_a A[a,a]
  const z64* a; int lda;
  const z64* b; int ldb;
  int n;
  z64* out;
  const int* active;
};

// --------------------------------------------------------------- launchers
// Each launcher takes device arrays of descriptors plus the host-known grid
// sizes; all are asynchronous on `st`.
// variant: tile shape (0: 64 x 64, 1: 16 x 256, 2: 256 x 16); tile_start
// must be built with zgemm_tiles of the same variant.
void launch_zgemm(const GemmDesc* d, const int* tile_start, int nprob, int total_tiles,
                  cudaStream_t st, int variant = 0);
int zgemm_tiles(int m, int n, int variant = 0);  // CTAs one problem needs
int zgemm_variant(const std::vector<GemmDesc>& ds);  // tile shape padding the group least
int zgemm_num_variants();

void launch_zform(const FormDesc* d, const int* tile_start, int nprob, int total_tiles,
                  cudaStream_t st);
int zform_tiles(int rows, int cols);

// Panel width used for a group whose largest block is smax (keeps the
// register-resident panel kernel within 32 complex values per thread).
int lu_panel_width(int smax);
// tournament != 0: tournament pivoting on the 8-CTA cluster panels (two cluster
// barriers per panel instead of one per column); others use partial pivoting.
void launch_lu_panel(const LuDesc* d, int nprob, int k0, int nb, int smax, cudaStream_t st, int tournament = 0);
// nbo > 0: two-level blocking with outer width nbo (the solve stops at the
// outer block's end); far: the column ranges and row exchanges (see
// lu_rowblock_kernel); far 3 (every row exchange of the outer block on the
// columns right of it) runs as one gather per column when its staging fits.
// max_rows: the largest block s of the group.
void launch_lu_rowblock(const LuDesc* d, int nprob, int k0, int nb, int nbo, int far, int max_cols,
                        cudaStream_t st, int max_rows = 0);
void launch_lu_backsub_diag(const LuDesc* d, int nprob, int k0, int nb, int max_rhs,
                            cudaStream_t st);
// Hermitian LDL^H panel without pivoting (see ss_lu.cu); smax: largest block of the group.
void launch_herm_panel(const LuDesc* d, int nprob, int k0, int nb, int smax, cudaStream_t st);

void launch_norm1(const Norm1Desc* d, int nprob, int max_cols, cudaStream_t st);
void launch_trace(const TraceDesc* d, int nprob, cudaStream_t st);

// Doubling convergence: active problems add `count` to iters, then drop out
// when max(n_a, n_b) <= tol * n_d, at the cap, or on NaN; resets n_a, n_b.
void launch_decim_check(double* na, double* nb, const double* nd, int* act, int* iters,
                        int* conv, int nprob, double tol, int cap, int count, cudaStream_t st);

void launch_fill_i32(int* p, int n, int v, cudaStream_t st);

}  // namespace ss
struct ss_mlp;
namespace ss {
cudaStream_t mlp_stream(const ss_mlp* n);
void mlp_dims(const ss_mlp* n, int* n_in, int* n_out, int* max_batch);
void launch_real_part(const z64* in, double* out, int n, cudaStream_t st);
// out[i] = scale * Im(in[i])
void launch_scaled_imag(const z64* in, double* out, int n, double scale, cudaStream_t st);
// out += sum |a|^2 (Norm1Desc reused; *out must start at 0)
void launch_frob2(const Norm1Desc* d, int nprob, int max_cols, cudaStream_t st);
void launch_unpack_g(const float* y, int s, double inv_scale, z64* g, int ldg, cudaStream_t st);

// Descriptors of the Caroli trace T = Re Tr[Gamma_L G Gamma_R G^H] for n_pts
// points of size s, with scratch laid out as [GamL | GamR | M1 | M2] per point
// (4 s^2 complex) followed by n_pts complex traces.  Fills the host vectors.
void caroli_descriptors(int n_pts, int s, const z64* sigL, const z64* sigR, const z64* G, z64* scratch,
                        std::vector<FormDesc>& f, std::vector<GemmDesc>& g, std::vector<TraceDesc>& t);
size_t caroli_scratch_elems(int n_pts, int s);

}  // namespace ss
