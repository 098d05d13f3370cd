// FP64 dense linear algebra for the projectors: thin Householder QR of a
// tall-skinny N x k block and one-sided (Hestenes) Jacobi SVD of a small
// k x k matrix.  Both keep the columns they work on as contiguous rows of a
// transposed copy, so every reflector / rotation touches contiguous memory.
// Each step is one launch; steps are ordered by the stream, so no kernel
// waits on another.
#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace ctm {
namespace {

constexpr int QR_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double t = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) t += sm[i];
    return t;
}

__device__ __forceinline__ double block_max(double v, double* sm) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double t = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) t = fmax(t, sm[i]);
    return t;
}

// Reflector of x = At[j][j:N] in the normalised form H = I - tau v v^T,
// v_j = 1, v_i = x_i / (x_j - beta), beta = -sign(x_j) |x|, tau in [1, 2]
// (the form of LAPACK's xLARFG): no quantity overflows when |x| is tiny.
// The norm is taken of x / max|x_i| so that squares do not underflow.
struct Reflector {
    double beta, tau, inv_denom;
};
__device__ Reflector make_reflector(const double* x, int j, int N, double* sm) {
    double mx = 0.0;
    for (int i = j + threadIdx.x; i < N; i += blockDim.x) mx = fmax(mx, fabs(x[i]));
    mx = block_max(mx, sm);
    Reflector r{x[j], 0.0, 0.0};
    if (mx == 0.0) return r;  // H = I
    const double inv = 1.0 / mx;
    double s2 = 0.0;
    for (int i = j + threadIdx.x; i < N; i += blockDim.x) {
        const double t = x[i] * inv;
        s2 = fma(t, t, s2);
    }
    s2 = block_sum(s2, sm);
    const double sig = mx * sqrt(s2);
    const double x0 = x[j];
    r.beta = (x0 >= 0.0) ? -sig : sig;
    const double denom = x0 - r.beta;  // |denom| = |x0| + sig >= sig > 0
    r.tau = (r.beta - x0) / r.beta;
    r.inv_denom = 1.0 / denom;
    return r;
}

// One Householder step j on At (k rows of length N, row c = column c).
// CTA b works on column c = j + b.  Every CTA recomputes the reflector of
// column j from At[j] (read-only in this launch); CTA 0 stores it.
__global__ void __launch_bounds__(QR_THREADS) k_house_step(double* __restrict__ At, double* __restrict__ V,
                                                           double* __restrict__ tau, double* __restrict__ beta,
                                                           double* __restrict__ R, int N, int k, int j) {
    __shared__ double sm[32];
    const int c = j + blockIdx.x;
    const double* x = At + (size_t)j * N;
    const Reflector rf = make_reflector(x, j, N, sm);
    if (blockIdx.x == 0) {
        double* v = V + (size_t)j * N;
        for (int i = threadIdx.x; i < N; i += blockDim.x)
            v[i] = (i < j) ? 0.0 : (i == j ? 1.0 : x[i] * rf.inv_denom);
        if (threadIdx.x == 0) { tau[j] = rf.tau; beta[j] = rf.beta; }
        return;
    }
    if (rf.tau == 0.0) {
        if (threadIdx.x == 0) R[(size_t)j * k + c] = At[(size_t)c * N + j];
        return;
    }
    double* a = At + (size_t)c * N;
    double w = 0.0;
    for (int i = j + threadIdx.x; i < N; i += blockDim.x) w = fma(i == j ? 1.0 : x[i] * rf.inv_denom, a[i], w);
    w = block_sum(w, sm) * rf.tau;
    for (int i = j + threadIdx.x; i < N; i += blockDim.x) a[i] -= w * (i == j ? 1.0 : x[i] * rf.inv_denom);
    // thread 0 owns index j in the strided loop, so it reads its own update
    if (threadIdx.x == 0) R[(size_t)j * k + c] = a[j];
}

// Q accumulation step j: Qt rows c >= j  <-  (I - tau v v^T) Qt[c].
__global__ void __launch_bounds__(QR_THREADS) k_house_apply(double* __restrict__ Qt, const double* __restrict__ V,
                                                            const double* __restrict__ tau, int N, int j) {
    __shared__ double sm[32];
    const double t = tau[j];
    if (t == 0.0) return;
    const int c = j + blockIdx.x;
    const double* v = V + (size_t)j * N;
    double* q = Qt + (size_t)c * N;
    double w = 0.0;
    for (int i = j + threadIdx.x; i < N; i += blockDim.x) w = fma(v[i], q[i], w);
    w = block_sum(w, sm) * t;
    for (int i = j + threadIdx.x; i < N; i += blockDim.x) q[i] -= w * v[i];
}

__global__ void k_eye_rows(double* __restrict__ Qt, int N, int k) {
    const size_t total = (size_t)k * N;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / N), i = (int)(t % N);
        Qt[t] = (i == c) ? 1.0 : 0.0;
    }
}

// Q[i][c] = sgn_c Qt[c][i];  R rows scaled by sgn_j, diagonal |beta_j|, lower part 0.
__global__ void k_qr_out(const double* __restrict__ Qt, const double* __restrict__ alpha,
                         const double* __restrict__ Rtmp, double* __restrict__ Q, double* __restrict__ R, int N,
                         int k) {
    const size_t totalQ = (size_t)N * k;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < totalQ; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / k), c = (int)(t % k);
        const double sg = alpha[c] < 0.0 ? -1.0 : 1.0;
        Q[t] = sg * Qt[(size_t)c * N + i];
    }
    const size_t totalR = (size_t)k * k;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < totalR; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / k), c = (int)(t % k);
        const double sg = alpha[j] < 0.0 ? -1.0 : 1.0;
        double v = 0.0;
        if (c == j) v = fabs(alpha[j]);
        else if (c > j) v = sg * Rtmp[t];
        R[t] = v;
    }
}

inline unsigned grid_for(size_t n, unsigned threads = 256) {
    size_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    if (b == 0) b = 1;
    return (unsigned)b;
}

// ---------------------------------------------------------------------------
// one-sided Jacobi.  Gt/Wt: nb matrices of k rows (row c = column c).
// Round r of the round-robin schedule pairs positions p and n-1-p with
// pos(0) = 0, pos(i) = 1 + (i - 1 + r) mod (n - 1), n = k rounded up to even.
// One warp per pair.  off[sweep*nb + b] collects max |g_p.g_q|/(|g_p||g_q|);
// a sweep whose predecessor was already below tol does nothing.
// ---------------------------------------------------------------------------
__global__ void k_jacobi_round(double* __restrict__ Gt, double* __restrict__ Wt, int k, int n, int r, int sweep,
                               unsigned long long* __restrict__ off, double tol) {
    const int b = blockIdx.y, nb = gridDim.y;
    if (sweep > 0 && __longlong_as_double((long long)off[(size_t)(sweep - 1) * nb + b]) < tol) return;
    const int p = blockIdx.x;
    auto pos = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + r) % (n - 1); };
    int P = pos(p), Q = pos(n - 1 - p);
    if (P >= k || Q >= k) return;
    if (P > Q) { const int t = P; P = Q; Q = t; }
    double* g = Gt + (size_t)b * k * k;
    double* gp = g + (size_t)P * k;
    double* gq = g + (size_t)Q * k;
    double a = 0.0, bb = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < k; i += 32) {
        const double x = gp[i], y = gq[i];
        a = fma(x, x, a);
        bb = fma(y, y, bb);
        c = fma(x, y, c);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        bb += __shfl_xor_sync(0xffffffffu, bb, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (a == 0.0 || bb == 0.0) return;
    const double rel = fabs(c) / (sqrt(a) * sqrt(bb));
    if (threadIdx.x == 0) atomicMax(off + (size_t)sweep * nb + b, (unsigned long long)__double_as_longlong(rel));
    if (!(rel > tol)) return;
    const double z = (bb - a) / (2.0 * c);
    const double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
    const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
    for (int i = threadIdx.x; i < k; i += 32) {
        const double x = gp[i], y = gq[i];
        gp[i] = cs * x - sn * y;
        gq[i] = sn * x + cs * y;
    }
    if (Wt) {
        double* w = Wt + (size_t)b * k * k;
        double* wp = w + (size_t)P * k;
        double* wq = w + (size_t)Q * k;
        for (int i = threadIdx.x; i < k; i += 32) {
            const double x = wp[i], y = wq[i];
            wp[i] = cs * x - sn * y;
            wq[i] = sn * x + cs * y;
        }
    }
}

// sigma_c = |g_c|; rank = position in descending order (ties by index).
__global__ void k_jacobi_finish(const double* __restrict__ Gt, const double* __restrict__ Wt, int k,
                                double* __restrict__ U, double* __restrict__ S, double* __restrict__ V) {
    extern __shared__ double sig[];
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(Gt[(size_t)c * k + i], Gt[(size_t)c * k + i], s);
        sig[c] = sqrt(s);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        const double sc = sig[c];
        int rank = 0;
        for (int c2 = 0; c2 < k; ++c2) rank += (sig[c2] > sc) || (sig[c2] == sc && c2 < c);
        S[rank] = sc;
        const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
        for (int i = 0; i < k; ++i) {
            U[(size_t)i * k + rank] = Gt[(size_t)c * k + i] * inv;
            V[(size_t)i * k + rank] = Wt[(size_t)c * k + i];
        }
    }
}

__global__ void k_svals_finish(const double* __restrict__ Gt, int k, double* __restrict__ out) {
    extern __shared__ double sig[];
    const int b = blockIdx.x;
    const double* g = Gt + (size_t)b * k * k;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(g[(size_t)c * k + i], g[(size_t)c * k + i], s);
        sig[c] = sqrt(s);
    }
    __syncthreads();
    double tot = 0.0;
    for (int c = 0; c < k; ++c) tot += sig[c];
    const double inv = tot > 0.0 ? 1.0 / tot : 0.0;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        const double sc = sig[c];
        int rank = 0;
        for (int c2 = 0; c2 < k; ++c2) rank += (sig[c2] > sc) || (sig[c2] == sc && c2 < c);
        out[(size_t)b * k + rank] = sc * inv;
    }
}

__global__ void k_eye_batch(double* __restrict__ W, int k, int nb) {
    const size_t total = (size_t)nb * k * k;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t rem = t % ((size_t)k * k);
        W[t] = (rem / k == rem % k) ? 1.0 : 0.0;
    }
}

// batched transpose of nb k x k matrices
__global__ void k_transpose_batch(const double* __restrict__ A, double* __restrict__ At, int k, int nb) {
    const size_t total = (size_t)nb * k * k;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t b = t / ((size_t)k * k), rem = t % ((size_t)k * k);
        const size_t i = rem / k, j = rem % k;
        At[b * k * k + j * k + i] = A[t];
    }
}

constexpr int JACOBI_MAX_SWEEPS = 12;
constexpr double JACOBI_TOL = 1e-15;

}  // namespace

// ---------------------------------------------------------------------------
size_t qr_ws_bytes(int N, int k) {
    return sizeof(double) * (3 * (size_t)k * N + (size_t)k * k + 2 * (size_t)k) + 256;
}

cudaError_t qr(const double* Y, int N, int k, double* Q, double* R, void* ws, cudaStream_t s) {
    if (N < k || k <= 0) return cudaErrorInvalidValue;
    double* At = (double*)ws;
    double* V = At + (size_t)k * N;
    double* Qt = V + (size_t)k * N;
    double* Rtmp = Qt + (size_t)k * N;
    double* tau = Rtmp + (size_t)k * k;
    double* alpha = tau + k;  // diagonal of R before the sign fix
    const int dims[2] = {N, k}, perm[2] = {1, 0};
    cudaError_t e = permute(Y, At, 2, dims, perm, s);
    if (e) return e;
    for (int j = 0; j < k; ++j) {
        ++g_launches;
        k_house_step<<<k - j, QR_THREADS, 0, s>>>(At, V, tau, alpha, Rtmp, N, k, j);
    }
    ++g_launches;
    k_eye_rows<<<grid_for((size_t)k * N), 256, 0, s>>>(Qt, N, k);
    for (int j = k - 1; j >= 0; --j) {
        ++g_launches;
        k_house_apply<<<k - j, QR_THREADS, 0, s>>>(Qt, V, tau, N, j);
    }
    ++g_launches;
    k_qr_out<<<grid_for((size_t)N * k), 256, 0, s>>>(Qt, alpha, Rtmp, Q, R, N, k);
    return cudaGetLastError();
}

size_t svd_ws_bytes(int k) {
    return sizeof(double) * 2 * (size_t)k * k + sizeof(unsigned long long) * JACOBI_MAX_SWEEPS + 256;
}

cudaError_t svd(const double* G, int k, double* U, double* S, double* V, void* ws, cudaStream_t s) {
    if (k <= 0 || k > 1024) return cudaErrorInvalidValue;
    double* Gt = (double*)ws;
    double* Wt = Gt + (size_t)k * k;
    unsigned long long* off = (unsigned long long*)(Wt + (size_t)k * k);
    cudaError_t e = cudaMemsetAsync(off, 0, sizeof(unsigned long long) * JACOBI_MAX_SWEEPS, s);
    if (e) return e;
    ++g_launches;
    k_transpose_batch<<<grid_for((size_t)k * k), 256, 0, s>>>(G, Gt, k, 1);
    ++g_launches;
    k_eye_batch<<<grid_for((size_t)k * k), 256, 0, s>>>(Wt, k, 1);
    const int n = k + (k & 1);
    for (int sw = 0; sw < JACOBI_MAX_SWEEPS; ++sw)
        for (int r = 0; r < n - 1; ++r) {
            ++g_launches;
            k_jacobi_round<<<dim3(n / 2, 1), 32, 0, s>>>(Gt, Wt, k, n, r, sw, off, JACOBI_TOL);
        }
    ++g_launches;
    k_jacobi_finish<<<1, 256, sizeof(double) * k, s>>>(Gt, Wt, k, U, S, V);
    return cudaGetLastError();
}

size_t svals_ws_bytes(int k, int nb) {
    return sizeof(double) * (size_t)nb * k * k + sizeof(unsigned long long) * JACOBI_MAX_SWEEPS * nb + 256;
}

cudaError_t svals_normalised(const double* Gs, int k, int nb, double* out, void* ws, cudaStream_t s) {
    if (k <= 0 || k > 1024 || nb <= 0 || nb > 65535) return cudaErrorInvalidValue;
    double* Gt = (double*)ws;
    unsigned long long* off = (unsigned long long*)(Gt + (size_t)nb * k * k);
    cudaError_t e = cudaMemsetAsync(off, 0, sizeof(unsigned long long) * JACOBI_MAX_SWEEPS * nb, s);
    if (e) return e;
    ++g_launches;
    k_transpose_batch<<<grid_for((size_t)nb * k * k), 256, 0, s>>>(Gs, Gt, k, nb);
    const int n = k + (k & 1);
    for (int sw = 0; sw < JACOBI_MAX_SWEEPS; ++sw)
        for (int r = 0; r < n - 1; ++r) {
            ++g_launches;
            k_jacobi_round<<<dim3(n / 2, nb), 32, 0, s>>>(Gt, nullptr, k, n, r, sw, off, JACOBI_TOL);
        }
    ++g_launches;
    k_svals_finish<<<nb, 256, sizeof(double) * k, s>>>(Gt, k, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free SVD: the same Jacobi SVD with its scratch in a file-scope
// device array.  The array's name in host code is only a host-side stand-in,
// so the device address is looked up once per device with
// cudaGetSymbolAddress (the first call on a device does this, with that
// device current) and passed to the kernels like any other workspace.
// ---------------------------------------------------------------------------
namespace {
constexpr int SVD_NOALLOC_MAX_K = 256;
constexpr size_t SVD_NOALLOC_BYTES =
    sizeof(double) * 2 * (size_t)SVD_NOALLOC_MAX_K * SVD_NOALLOC_MAX_K +
    sizeof(unsigned long long) * JACOBI_MAX_SWEEPS + 256;
static __device__ __align__(256) unsigned char g_svd_scratch[SVD_NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};
}  // namespace

int svd_noalloc_max_k() { return SVD_NOALLOC_MAX_K; }

cudaError_t svd_noalloc(const double* G, int k, double* U, double* S, double* V, cudaStream_t s) {
    if (k <= 0 || k > SVD_NOALLOC_MAX_K) return cudaErrorInvalidValue;
    static_assert(SVD_NOALLOC_BYTES >= sizeof(double) * 2 * (size_t)SVD_NOALLOC_MAX_K * SVD_NOALLOC_MAX_K +
                                           sizeof(unsigned long long) * JACOBI_MAX_SWEEPS,
                  "scratch holds the Jacobi workspace of the largest k");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    void* ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_svd_scratch);
            if (e != cudaSuccess) return e;
            g_scratch_ptr[dev] = p;
        }
        ws = g_scratch_ptr[dev];
    }
    return svd(G, k, U, S, V, ws, s);
}

}  // namespace ctm
