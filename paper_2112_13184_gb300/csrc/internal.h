// Internal declarations shared by the libctm translation units.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include <cstdint>

#include "ctm.h"

namespace ctm {

// kernel launches issued by this library (process-wide, all handles and
// host threads)
extern std::atomic<long long> g_launches;

// ---- launch wrappers (kernels.cu) ----------------------------------------
// All return cudaGetLastError() of their launch; work on `s`.
// ws (optional): split-K partials when the output has few tiles and K is long;
// dgemm_splitk_ws_doubles gives the size it wants (0 = no split).
size_t dgemm_splitk_ws_doubles(int M, int N, int K);
cudaError_t dgemm(bool tA, bool tB, int M, int N, int K, double alpha, const double* A, int lda,
                  const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t s,
                  double* ws = nullptr, size_t ws_doubles = 0);
cudaError_t permute(const double* src, double* dst, int ndim, const int* dims, const int* perm,
                    cudaStream_t s);
// X[r*ld + c] *= w[c], r < rows, c < cols
cudaError_t scale_cols(double* X, int rows, int cols, int ld, const double* w, cudaStream_t s);
// dst[i][j] += src[i][j], i < rows, j < cols (row strides lds, ldd)
cudaError_t add_block(const double* src, int rows, int cols, int lds, double* dst, int ldd, cudaStream_t s);
// w[j] = s[j] > cut*s[0] ? 1/sqrt(s[j]) : 0
cudaError_t inv_sqrt_cut(const double* sv, double* w, int n, double cut, cudaStream_t s);
// bits of max|x| into *maxbits (must be zeroed first); sticky
cudaError_t maxabs(const double* x, size_t n, unsigned long long* maxbits, cudaStream_t s);
// x /= max; sets *flag = 1 if max is not finite, 2 (when still 0) if max is 0
cudaError_t scale_by_max(double* x, size_t n, const unsigned long long* maxbits, int* flag,
                         cudaStream_t s);
// *out = sum_i x[i] y[i] in a fixed order; ws: dot_ws_doubles() doubles
size_t dot_ws_doubles();
cudaError_t dot(const double* x, const double* y, size_t n, double* out, double* ws, cudaStream_t s);
// out[m] = trace of the m-th n x n matrix of As (contiguous), m < nm
cudaError_t traces(const double* As, int n, int nm, double* out, cudaStream_t s);
// blocks x threads threads, each 8 x iters FP64 FMAs; out: blocks x threads doubles
cudaError_t dfma_probe(double* out, int blocks, int threads, int iters, cudaStream_t s);
// T[a,k,k',b] (chi x D x D x chi) symmetrised over (k, k') in place
cudaError_t sym_kk(double* T, int chi, int D, cudaStream_t s);
// out[i] = standard normal, Philox4x32-10 counter (seed, stream_id, i)
cudaError_t rng_normal(double* out, size_t n, uint64_t seed, uint64_t stream_id, cudaStream_t s);

// ---- dense linear algebra (linalg.cu) ---------------------------------------
size_t qr_ws_bytes(int N, int k);
// Thin Householder QR.  One persistent cooperative launch when the row
// slabs fit in shared memory (every grid barrier bounded: on a time-out *err
// -- or, without err, the first int of ws -- becomes 1 and Q, R are not
// valid), else two launches per column step.
cudaError_t qr(const double* Y, int N, int k, double* Q, double* R, void* ws, cudaStream_t s, int* err = nullptr);
size_t svd_ws_bytes(int k);
// *status (optional; else the first int of ws) becomes 1 when the Jacobi
// iteration still rotated in its last allowed sweep
cudaError_t svd(const double* G, int k, double* U, double* S, double* V, void* ws, cudaStream_t s,
                int* status = nullptr);
// two independent SVDs of k x k matrices in one Jacobi launch (one cluster
// each); ws: svd2_ws_bytes(k); *status as for svd()
size_t svd2_ws_bytes(int k);
cudaError_t svd2(const double* G0, const double* G1, int k, double* U0, double* S0, double* V0, double* U1,
                 double* S1, double* V1, void* ws, cudaStream_t s, int* status = nullptr);
// svd() with its workspace in a static device array (k <= svd_noalloc_max_k())
int svd_noalloc_max_k();
cudaError_t svd_noalloc(const double* G, int k, double* U, double* S, double* V, cudaStream_t s);
// eigenvalues of a small real m x m matrix (m <= small_eig_max(), row stride
// ldh): out[4m] = Re(l_i / l_0), Im(l_i / l_0), |l_i|, -ln|l_i / l_0| / period,
// sorted by |l_i| descending; *status (optional) 0, 1 = QR iteration cap hit,
// 2 = all eigenvalues zero
int small_eig_max();
cudaError_t small_eig(const double* H, int m, int ldh, double period, double* out, int* status, cudaStream_t s,
                      double* ev = nullptr);
// real basis of the Ritz vectors of the leading eigenvalues of H (m x m,
// row stride ldh): ev = small_eig's sorted eigenvalues (re, im pairs);
// Y[j][0..m) for j < nvec holds Re y_i of a real eigenvalue, or Re y_i and
// Im y_i of a complex pair (its conjugate skipped), y_i by inverse iteration
cudaError_t ritz_basis(const double* H, int m, int ldh, const double* ev, int nvec, double* Y, cudaStream_t s);
// singular values only (descending) of a batch of nb k x k matrices, each
// normalised to sum 1; Gs contiguous, out nb*k
size_t svals_ws_bytes(int k, int nb);
cudaError_t svals_normalised(const double* Gs, int k, int nb, double* out, void* ws, cudaStream_t s);

// ---- emulated-FP64 GEMM on the tensor cores (ozaki.cu) ----------------------
// strided multi-index view (row-major over dim[0..n-1])
struct OzView {
    int n;
    int dim[4];
    long long stride[4];
};
// Split an R x K FP64 operand (element (r,k) at X[r*rs + k*cs]) into s BF16
// slices [s][R][K8] plus per-row exponents, in a buffer of oz_split_bytes.
size_t oz_split_bytes(int R, int K, int s);
cudaError_t oz_split(const double* X, int R, int K, long long rs, long long cs, int s, void* buf, cudaStream_t st);
// element (r, k) at X[view(rv, r) + view(kv, k)]
cudaError_t oz_split_view(const double* X, int R, int K, const OzView& rv, const OzView& kv, int s, void* buf,
                          cudaStream_t st);
// TF32 operand slices of 3xTF32 (two FP32-stored TF32 slices per element)
size_t oz_split_tf32_bytes(int R, int K);
cudaError_t oz_split_tf32(const double* X, int R, int K, const OzView& rv, const OzView& kv, void* buf,
                          cudaStream_t st);
// C[M,N] = alpha A B + beta C from split A (M rows) and split B (N rows = columns of B).
// mode 0: exact-level emulated FP64 (s slices); 1: split-BF16, FP32 accumulation
// (s = 3 BF16 slices); 2: 3xTF32, FP32 accumulation (s = 2 TF32 slices)
size_t oz_gemm_ws_bytes(int M, int N, int K, int s, int mode = 0);
cudaError_t oz_gemm(int M, int N, int K, int s, const void* Asplit, const void* Bsplit, double alpha, double beta,
                    double* C, int ldc, void* ws, size_t ws_bytes, int* err, cudaStream_t st, int mode = 0);
// C written at C[view(out_r, m) + view(out_c, n)]
cudaError_t oz_gemm_view(int M, int N, int K, int s, const void* Asplit, const void* Bsplit, double alpha,
                         double beta, double* C, const OzView& out_r, const OzView& out_c, void* ws, size_t ws_bytes,
                         int* err, cudaStream_t st, int mode = 0);

// Failure-detection check of the bounded mbarrier wait used by the tensor-core
// GEMM: one thread waits at most limit_cycles on a barrier that receives an
// arrival only when `arrive` is set; *err becomes 1 when the wait gave up.
cudaError_t wait_probe(long long limit_cycles, int arrive, int* err, cudaStream_t st);

}  // namespace ctm
