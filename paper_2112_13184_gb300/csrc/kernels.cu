// FP64 building blocks of the CTMRG sweep: GEMM, axis permutation,
// normalisation, counter-based Gaussian numbers.  GB300 (sm_103a).
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace ctm {

std::atomic<long long> g_launches{0};

// ---------------------------------------------------------------------------
// FP64 GEMM, row-major: C[M,N] = alpha op(A) op(B) + beta C.
// 64x64 tile, K-step 16, 256 threads, 4x4 outputs per thread strided by 16
// so that shared-memory reads broadcast without bank conflicts.  On GB300
// the FP64 pipe, not memory, bounds this kernel.
// ---------------------------------------------------------------------------
namespace {
constexpr int GB = 64, GK = 16;

// Split-K: blockIdx.z takes K range [z*kchunk, (z+1)*kchunk) and writes its
// partial product (alpha=1, beta=0) to C + z*zstride; a second kernel sums
// the partials in fixed order, so results do not depend on scheduling.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha,
                                               const double* __restrict__ A, int lda,
                                               const double* __restrict__ B, int ldb, double beta,
                                               double* __restrict__ C, int ldc, int kchunk, size_t zstride) {
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    C += blockIdx.z * zstride;
    __shared__ double As[GK][GB + 1];
    __shared__ double Bs[GK][GB + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long m0 = (long long)blockIdx.x * GB, n0 = (long long)blockIdx.y * GB;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += GK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = tid + 256 * r;
            int mm, kk;
            if (!TA) { mm = idx >> 4; kk = idx & 15; } else { mm = idx & 63; kk = idx >> 6; }
            const long long gm = m0 + mm;
            const int gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < kend) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            As[kk][mm] = v;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = tid + 256 * r;
            int nn, kk;
            if (!TB) { nn = idx & 63; kk = idx >> 6; } else { nn = idx >> 4; kk = idx & 15; }
            const long long gn = n0 + nn;
            const int gk = k0 + kk;
            double v = 0.0;
            if (gn < N && gk < kend) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            double* c = C + (size_t)gm * ldc + gn;
            const double v = alpha * acc[i][j];
            *c = (beta == 0.0) ? v : fma(beta, *c, v);
        }
    }
}
__global__ void k_splitk_reduce(const double* __restrict__ P, int splits, int M, int N, double alpha,
                                double beta, double* __restrict__ C, int ldc) {
    const size_t total = (size_t)M * N;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int z = 0; z < splits; ++z) acc += P[(size_t)z * total + t];
        const size_t r = t / N, c = t % N;
        double* cp = C + r * ldc + c;
        *cp = (beta == 0.0) ? alpha * acc : fma(beta, *cp, alpha * acc);
    }
}

template <bool TA, bool TB>
void launch(dim3 g, cudaStream_t s, int M, int N, int K, double alpha, const double* A, int lda, const double* B,
            int ldb, double beta, double* C, int ldc, int kchunk, size_t zs) {
    ++g_launches;
    k_dgemm<TA, TB><<<g, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kchunk, zs);
}
}  // namespace

size_t dgemm_splitk_ws_doubles(int M, int N, int K) {
    const long long tiles = (long long)((M + GB - 1) / GB) * ((N + GB - 1) / GB);
    if (tiles >= 152 || K < 512) return 0;
    long long splits = std::min<long long>((304 + tiles - 1) / tiles, K / 256);
    if (splits < 2) return 0;
    return (size_t)splits * M * N;
}

cudaError_t dgemm(bool tA, bool tB, int M, int N, int K, double alpha, const double* A, int lda,
                  const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t s, double* ws,
                  size_t ws_doubles) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((M + GB - 1) / GB), (unsigned)((N + GB - 1) / GB), 1);
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    const size_t need = dgemm_splitk_ws_doubles(M, N, K);
    int splits = 1, kchunk = K > 0 ? K : 1;
    double* out = C;
    int ldo = ldc;
    double a = alpha, b = beta;
    if (need && ws && need <= ws_doubles) {
        splits = (int)(need / ((size_t)M * N));
        kchunk = ((K + splits - 1) / splits + GK - 1) / GK * GK;
        splits = (K + kchunk - 1) / kchunk;
        grid.z = splits;
        out = ws;
        ldo = N;
        a = 1.0;
        b = 0.0;
    }
    const size_t zs = (size_t)M * N;
    if (!tA && !tB) launch<false, false>(grid, s, M, N, K, a, A, lda, B, ldb, b, out, ldo, kchunk, zs);
    else if (tA && !tB) launch<true, false>(grid, s, M, N, K, a, A, lda, B, ldb, b, out, ldo, kchunk, zs);
    else if (!tA && tB) launch<false, true>(grid, s, M, N, K, a, A, lda, B, ldb, b, out, ldo, kchunk, zs);
    else launch<true, true>(grid, s, M, N, K, a, A, lda, B, ldb, b, out, ldo, kchunk, zs);
    if (splits > 1) {
        size_t blocks = (zs + 255) / 256;
        if (blocks > 152 * 8) blocks = 152 * 8;
        ++g_launches;
        k_splitk_reduce<<<(unsigned)blocks, 256, 0, s>>>(ws, splits, M, N, alpha, beta, C, ldc);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Axis permutation.  One thread per destination element (coalesced writes);
// the source offset comes from the destination multi-index.
// ---------------------------------------------------------------------------
namespace {
struct PermArgs {
    int ndim;
    unsigned dims[8];     // destination dims
    unsigned stride[8];   // source stride of each destination axis
};

__global__ void k_permute32(const double* __restrict__ src, double* __restrict__ dst, unsigned total,
                            PermArgs p) {
    for (unsigned o = blockIdx.x * blockDim.x + threadIdx.x; o < total; o += gridDim.x * blockDim.x) {
        unsigned rem = o, off = 0;
        for (int a = p.ndim - 1; a >= 0; --a) {
            const unsigned i = rem % p.dims[a];
            rem /= p.dims[a];
            off += i * p.stride[a];
        }
        dst[o] = __ldg(src + off);
    }
}
}  // namespace

cudaError_t permute(const double* src, double* dst, int ndim, const int* dims, const int* perm,
                    cudaStream_t s) {
    if (ndim < 1 || ndim > 8) return cudaErrorInvalidValue;
    unsigned long long sstride[8];
    unsigned long long total = 1;
    for (int a = ndim - 1; a >= 0; --a) {
        sstride[a] = total;
        total *= (unsigned long long)dims[a];
    }
    if (total == 0) return cudaSuccess;
    if (total >= (1ull << 32)) return cudaErrorInvalidValue;
    PermArgs p;
    p.ndim = ndim;
    for (int a = 0; a < ndim; ++a) {
        p.dims[a] = (unsigned)dims[perm[a]];
        p.stride[a] = (unsigned)sstride[perm[a]];
    }
    const unsigned threads = 256;
    unsigned long long blocks = (total + threads - 1) / threads;
    if (blocks > 152ull * 64) blocks = 152ull * 64;
    ++g_launches;
    k_permute32<<<(unsigned)blocks, threads, 0, s>>>(src, dst, (unsigned)total, p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// elementwise helpers
// ---------------------------------------------------------------------------
namespace {
__global__ void k_scale_cols(double* X, int rows, int cols, int ld, const double* __restrict__ w) {
    const size_t total = (size_t)rows * cols;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        X[(size_t)r * ld + c] *= w[c];
    }
}
__global__ void k_inv_sqrt_cut(const double* __restrict__ sv, double* __restrict__ w, int n, double cut) {
    const double s0 = sv[0];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double v = sv[j];
        w[j] = (s0 > 0.0 && v > cut * s0) ? 1.0 / sqrt(v) : 0.0;
    }
}
__global__ void k_maxabs(const double* __restrict__ x, size_t n, unsigned long long* maxbits) {
    double m = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double a = fabs(x[i]);
        // NaN compares false: force it through as the largest bit pattern
        m = (a > m || a != a) ? a : m;
    }
    unsigned long long b = __double_as_longlong(m);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = t > b ? t : b;
    }
    __shared__ unsigned long long sm[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sm[w] = b;
    __syncthreads();
    if (w == 0) {
        b = (lane < (int)(blockDim.x >> 5)) ? sm[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
            b = t > b ? t : b;
        }
        if (lane == 0) atomicMax(maxbits, b);
    }
}
__global__ void k_scale_by_max(double* x, size_t n, const unsigned long long* maxbits, int* flag) {
    const unsigned long long b = *maxbits;
    if (b >= 0x7ff0000000000000ull) {  // Inf or NaN
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(flag, 1);
        return;
    }
    const double m = __longlong_as_double((long long)b);
    if (m == 0.0) {  // an all-zero tensor: the projectors have collapsed
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(flag, 0, 2);
        return;
    }
    const double inv = 1.0 / m;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] *= inv;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the
// published definition: 10 rounds of two 32x32->64 multiplies with the
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += W0; k.y += W1; }
        const unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}
__global__ void k_rng_normal(double* __restrict__ out, size_t n, uint64_t seed, uint64_t sid) {
    const size_t pairs = (n + 1) / 2;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < pairs; p += (size_t)gridDim.x * blockDim.x) {
        const uint4 r = philox4x32_10(make_uint4((unsigned)p, (unsigned)(p >> 32), (unsigned)sid, (unsigned)(sid >> 32)),
                                      make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
        // two 53-bit uniforms; u1 in (0, 1] for the logarithm
        const double u1 = 1.0 - (double)(((unsigned long long)(r.x >> 5) << 26) | (r.y >> 6)) * 0x1.0p-53;
        const double u2 = (double)(((unsigned long long)(r.z >> 5) << 26) | (r.w >> 6)) * 0x1.0p-53;
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        out[2 * p] = rad * cs;
        if (2 * p + 1 < n) out[2 * p + 1] = rad * sn;
    }
}
// Dot product in two passes with a fixed grid, so the summation order (and
// the result) does not depend on scheduling: pass 1 leaves one partial per
// block, pass 2 (one block) adds them in block order.
constexpr int DOT_BLOCKS = 152 * 4;
__global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y, size_t n,
                              double* __restrict__ part) {
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc = fma(x[i], y[i], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double sm[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sm[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sm[i];
        part[blockIdx.x] = t;
    }
}
__global__ void k_dot_final(const double* __restrict__ part, int np, double* __restrict__ out) {
    __shared__ double sm[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) t += part[i];
    sm[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) s += sm[i];
        *out = s;
    }
}
// T[a,k,k',b] <- (T[a,k,k',b] + T[a,k',k,b]) / 2, one thread per pair k <= k'
__global__ void k_sym_kk(double* __restrict__ T, int chi, int D) {
    const size_t total = (size_t)chi * D * D * chi;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t b = t % chi, kk2 = (t / chi) % D, kk = (t / ((size_t)chi * D)) % D, a = t / ((size_t)chi * D * D);
        if (kk > kk2) continue;
        const size_t i1 = ((a * D + kk) * D + kk2) * chi + b, i2 = ((a * D + kk2) * D + kk) * chi + b;
        const double v = 0.5 * (T[i1] + T[i2]);
        T[i1] = v;
        T[i2] = v;
    }
}
inline unsigned grid_for(size_t n, unsigned threads = 256) {
    size_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    if (b == 0) b = 1;
    return (unsigned)b;
}
// dst[i][j] += src[i][j] for a rows x cols block (row strides lds, ldd)
__global__ void k_add_block(const double* __restrict__ src, int rows, int cols, int lds, double* __restrict__ dst,
                            int ldd) {
    const size_t total = (size_t)rows * cols;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / cols), j = (int)(t % cols);
        dst[(size_t)i * ldd + j] += src[(size_t)i * lds + j];
    }
}
}  // namespace

cudaError_t add_block(const double* src, int rows, int cols, int lds, double* dst, int ldd, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    ++g_launches;
    k_add_block<<<grid_for((size_t)rows * cols), 256, 0, s>>>(src, rows, cols, lds, dst, ldd);
    return cudaGetLastError();
}

cudaError_t scale_cols(double* X, int rows, int cols, int ld, const double* w, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    ++g_launches;
    k_scale_cols<<<grid_for((size_t)rows * cols), 256, 0, s>>>(X, rows, cols, ld, w);
    return cudaGetLastError();
}
cudaError_t inv_sqrt_cut(const double* sv, double* w, int n, double cut, cudaStream_t s) {
    ++g_launches;
    k_inv_sqrt_cut<<<1, 256, 0, s>>>(sv, w, n, cut);
    return cudaGetLastError();
}
cudaError_t maxabs(const double* x, size_t n, unsigned long long* maxbits, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ++g_launches;
    k_maxabs<<<grid_for(n), 256, 0, s>>>(x, n, maxbits);
    return cudaGetLastError();
}
cudaError_t scale_by_max(double* x, size_t n, const unsigned long long* maxbits, int* flag, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ++g_launches;
    k_scale_by_max<<<grid_for(n), 256, 0, s>>>(x, n, maxbits, flag);
    return cudaGetLastError();
}
// FP64 FMA throughput probe: every thread runs 8 independent FMA chains
// (enough in flight to keep the pipe busy); the result is stored so the
// chains are not optimised away.
__global__ void k_dfma_probe(double* __restrict__ out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = (double)(threadIdx.x + u) * 1e-3;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, b);
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += x[u];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// out[m] = trace of the n x n matrix As + m n^2, m < nm (one warp per matrix)
__global__ void k_traces(const double* __restrict__ As, int n, int nm, double* __restrict__ out) {
    const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (m >= nm) return;
    const double* a = As + (size_t)m * n * n;
    double t = 0.0;
    for (int i = lane; i < n; i += 32) t += a[(size_t)i * (n + 1)];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) out[m] = t;
}

size_t dot_ws_doubles() { return DOT_BLOCKS; }
cudaError_t dot(const double* x, const double* y, size_t n, double* out, double* ws, cudaStream_t s) {
    ++g_launches;
    k_dot_partial<<<DOT_BLOCKS, 256, 0, s>>>(x, y, n, ws);
    ++g_launches;
    k_dot_final<<<1, 256, 0, s>>>(ws, DOT_BLOCKS, out);
    return cudaGetLastError();
}
cudaError_t traces(const double* As, int n, int nm, double* out, cudaStream_t s) {
    ++g_launches;
    k_traces<<<(nm + 7) / 8, 256, 0, s>>>(As, n, nm, out);
    return cudaGetLastError();
}
cudaError_t dfma_probe(double* out, int blocks, int threads, int iters, cudaStream_t s) {
    ++g_launches;
    k_dfma_probe<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
    return cudaGetLastError();
}
cudaError_t sym_kk(double* T, int chi, int D, cudaStream_t s) {
    ++g_launches;
    k_sym_kk<<<grid_for((size_t)chi * D * D * chi), 256, 0, s>>>(T, chi, D);
    return cudaGetLastError();
}
cudaError_t rng_normal(double* out, size_t n, uint64_t seed, uint64_t sid, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ++g_launches;
    k_rng_normal<<<grid_for((n + 1) / 2), 256, 0, s>>>(out, n, seed, sid);
    return cudaGetLastError();
}

}  // namespace ctm
