// FP64 dense linear algebra for the projectors: thin Householder QR of a
// tall-skinny N x k block and one-sided (Hestenes) Jacobi SVD of a small
// k x k matrix.  Both keep the columns they work on as contiguous rows of a
// transposed copy, so every reflector / rotation touches contiguous memory.
// Each step is one launch; steps are ordered by the stream, so no kernel
// waits on another.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <algorithm>
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

// ---------------------------------------------------------------------------
// Householder QR, two launches per step over (row chunk x column) tiles so
// that every step uses the whole GPU.  Step j, phase A: every tile forms the
// partial dot x.a_c of the current column x = At[j] with a column a_c = At[c]
// (c = j gives |x|^2) over its rows.  Phase B: every tile reduces the
// partials in fixed order and applies the reflector in normalised form
// H = I - tau v v^T, v_j = 1, v_i = x_i / (x_j - beta), beta = -sign(x_j)|x|,
// tau = (beta - x_j)/beta in [1, 2], using v.a_c = (x.a_c - beta a_c[j]) /
// (x_j - beta).  a_c[j] is recorded in phase A, before phase B changes it.
// ---------------------------------------------------------------------------
constexpr int QR_CHUNK = 512;
constexpr int QR2_THREADS = 128;

__global__ void __launch_bounds__(QR2_THREADS) k_qr_dots(const double* __restrict__ At, int N, int k, int j,
                                                         double* __restrict__ P, double* __restrict__ Aj) {
    __shared__ double sm[32];
    const int ch = blockIdx.x, c = j + blockIdx.y;
    const int i0 = max(j, ch * QR_CHUNK), i1 = min(N, (ch + 1) * QR_CHUNK);
    const double* x = At + (size_t)j * N;
    const double* a = At + (size_t)c * N;
    double p = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) p = fma(x[i], a[i], p);
    p = block_sum(p, sm);
    if (threadIdx.x == 0) {
        P[(size_t)ch * k + c] = p;
        if (j >= ch * QR_CHUNK && j < (ch + 1) * QR_CHUNK) Aj[c] = a[j];
    }
}

__global__ void __launch_bounds__(QR2_THREADS) k_qr_update(double* __restrict__ At, double* __restrict__ V,
                                                           double* __restrict__ tau, double* __restrict__ beta,
                                                           double* __restrict__ R, int N, int k, int j, int nch,
                                                           const double* __restrict__ P,
                                                           const double* __restrict__ Aj) {
    const int ch = blockIdx.x, c = j + blockIdx.y;
    const int i0 = max(j, ch * QR_CHUNK), i1 = min(N, (ch + 1) * QR_CHUNK);
    const bool owns_j = j >= ch * QR_CHUNK && j < (ch + 1) * QR_CHUNK;
    double s2 = 0.0, xa = 0.0;
    for (int q = 0; q < nch; ++q) {
        s2 += P[(size_t)q * k + j];
        xa += P[(size_t)q * k + c];
    }
    const double xj = Aj[j];
    const double* x = At + (size_t)j * N;
    if (s2 == 0.0) {  // zero column: H = I
        if (c == j) {
            if (owns_j && threadIdx.x == 0) {
                V[(size_t)j * N + j] = 1.0;
                tau[j] = 0.0;
                beta[j] = xj;
            }
        } else if (owns_j && threadIdx.x == 0) {
            R[(size_t)j * k + c] = Aj[c];
        }
        return;
    }
    const double sig = sqrt(s2);
    const double bt = xj >= 0.0 ? -sig : sig;
    const double inv = 1.0 / (xj - bt);  // |xj - bt| = |xj| + sig >= sig > 0
    const double tu = (bt - xj) / bt;
    if (c == j) {
        double* v = V + (size_t)j * N;
        for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) v[i] = (i == j) ? 1.0 : x[i] * inv;
        if (owns_j && threadIdx.x == 0) {
            tau[j] = tu;
            beta[j] = bt;
        }
        return;
    }
    const double w = tu * (xa - bt * Aj[c]) * inv;
    double* a = At + (size_t)c * N;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) a[i] -= w * ((i == j) ? 1.0 : x[i] * inv);
    if (owns_j && threadIdx.x == 0) R[(size_t)j * k + c] = Aj[c] - w;
}

// Q accumulation step j: Qt rows c >= j  <-  (I - tau v v^T) Qt[c]
__global__ void __launch_bounds__(QR2_THREADS) k_qt_dots(const double* __restrict__ Qt, const double* __restrict__ V,
                                                         const double* __restrict__ tau, int N, int k, int j,
                                                         double* __restrict__ P) {
    __shared__ double sm[32];
    if (tau[j] == 0.0) return;
    const int ch = blockIdx.x, c = j + blockIdx.y;
    const int i0 = max(j, ch * QR_CHUNK), i1 = min(N, (ch + 1) * QR_CHUNK);
    const double* v = V + (size_t)j * N;
    const double* q = Qt + (size_t)c * N;
    double p = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) p = fma(v[i], q[i], p);
    p = block_sum(p, sm);
    if (threadIdx.x == 0) P[(size_t)ch * k + c] = p;
}

__global__ void __launch_bounds__(QR2_THREADS) k_qt_update(double* __restrict__ Qt, const double* __restrict__ V,
                                                           const double* __restrict__ tau, int N, int k, int j,
                                                           int nch, const double* __restrict__ P) {
    const double tu = tau[j];
    if (tu == 0.0) return;
    const int ch = blockIdx.x, c = j + blockIdx.y;
    const int i0 = max(j, ch * QR_CHUNK), i1 = min(N, (ch + 1) * QR_CHUNK);
    double d = 0.0;
    for (int q = 0; q < nch; ++q) d += P[(size_t)q * k + c];
    const double w = tu * d;
    const double* v = V + (size_t)j * N;
    double* qc = Qt + (size_t)c * N;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) qc[i] -= w * v[i];
}

// ---------------------------------------------------------------------------
// Householder QR in ONE persistent cooperative launch.  GB300 runs FP64 at
// about two DFMA per clock per SM, so the 2 N k^2 flops of each half (the
// factorisation and the explicit Q) are spread over every SM: CTA b holds
// rows [b nr, (b+1) nr) of the panel -- and later of Q -- in shared memory
// (column-major, rows contiguous), and every column step is
//   partial dots over the own rows -> one bounded grid barrier -> every
//   CTA adds the partials of all CTAs in the same fixed order (so all agree
//   on beta, tau and the update weights bit for bit, and a rerun gives the
//   same bits) -> reflector applied to the own rows,
// with the next column's partial dots fused behind the update: k barriers
// for the factorisation and k for Q = H_0 ... H_{k-1} [I; 0], accumulated
// backwards.  The reflector is the same normalised one as the per-step
// kernels above.  Partial sums and the published row j are double-buffered
// by step parity, so a CTA running ahead never overwrites what a slower one
// still reads.  Data written by other CTAs is read through L2 (ld.cg).
// ---------------------------------------------------------------------------
constexpr int PQR_THREADS = 256;
constexpr int PQR_MIN_ROWS = 16;
constexpr int PQR_MAX_GRID = 160;  // partials per column read by one CTA step (8 lanes x 20)
constexpr long long PQR_WAIT_CYCLES = 2000000000ll;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid-wide barrier of a cooperative launch (all CTAs resident).  Bounded:
// gives up after `limit` cycles, or at once when another CTA gave up,
// recording the failure in *err; returns false then, and the caller leaves.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nb, int* err,
                                             long long limit) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = atomicAdd(gen, 0u);
        __threadfence();
        if (atomicAdd(count, 1u) == nb - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*(volatile unsigned*)gen == g) {
                if (*(volatile int*)err) { ok = 0; break; }
                if (clock64() - t0 > limit) { atomicCAS(err, 0, 1); ok = 0; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok_s = ok && !*(volatile int*)err;
    }
    __syncthreads();
    return ok_s != 0;
}

__global__ void __launch_bounds__(PQR_THREADS) k_qr_persistent(const double* __restrict__ Y, int N, int k, int nr,
                                                               double* __restrict__ Q, double* __restrict__ R,
                                                               double* __restrict__ P, double* __restrict__ Ajg,
                                                               unsigned* bar, int* err, long long limit) {
    extern __shared__ double sm[];
    const int ld = nr | 1;                // odd column stride: a thread per column reads without bank conflicts
    double* S = sm;                       // panel slab [k][ld]: R above, reflectors below the diagonal
    double* Qs = S + (size_t)k * ld;      // Q slab [k][ld]
    double* tot = Qs + (size_t)k * ld;    // totals of the current step [k]
    double* wv = tot + k;                 // update weights [k]
    double* tau_s = wv + k;               // [k]
    double* beta_s = tau_s + k;           // [k]
    const int G = gridDim.x, cta = blockIdx.x;
    const int r0 = cta * nr, r1 = min(N, r0 + nr), nrl = max(0, r1 - r0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    unsigned* count = bar;
    unsigned* gen = bar + 1;

    for (int t = threadIdx.x; t < k * nr; t += blockDim.x) {
        const int c = t / nr, rl = t - c * nr;
        S[(size_t)c * ld + rl] = rl < nrl ? Y[(size_t)(r0 + rl) * k + c] : 0.0;
        Qs[(size_t)c * ld + rl] = (rl < nrl && r0 + rl == c) ? 1.0 : 0.0;
    }
    __syncthreads();

    // partial dots over the own rows >= j of column j (factor: x = column j;
    // Q: x = reflector j, 1 at row j) with the columns c >= j of `B`, stored
    // as this CTA's partials P[par][c][cta].  One thread per column sums its
    // rows in order: a shuffle tree over 32 lanes spent 5 FP64 adds per lane
    // on every column, more than the products themselves (nr ~ 54 rows)
    auto dots = [&](int j, int par, const double* B, bool reflector) {
        const int rl0 = max(0, j - r0);
        const double* x = S + (size_t)j * ld;
        const bool one_at_j = reflector && j >= r0 && j < r1;  // the reflector's implicit 1 is a row of this CTA
        for (int c = j + threadIdx.x; c < k; c += blockDim.x) {
            const double* a = B + (size_t)c * ld;
            double p = 0.0;
            int rl = rl0;
            if (one_at_j) p = a[rl++];
            for (; rl < nrl; ++rl) p = fma(x[rl], a[rl], p);
            P[((size_t)par * k + c) * G + cta] = p;
        }
    };
    // every CTA adds the G partials of each column c >= j in the same order:
    // 8 lanes per column, lane s takes partials s, s+8, ... (all its loads
    // issued before the first add), then a fixed 3-level shuffle tree
    auto read_totals = [&](int j, int s) {
        const int par = s & 1, sub = threadIdx.x & 7;
        for (int c0 = j; c0 < k; c0 += PQR_THREADS / 8) {
            const int c = c0 + (int)(threadIdx.x >> 3);
            double t = 0.0;
            if (c < k) {
                const double* pc = P + ((size_t)par * k + c) * G;
                double v[PQR_MAX_GRID / 8];
#pragma unroll
                for (int i = 0; i < PQR_MAX_GRID / 8; ++i) {
                    const int q = sub + 8 * i;
                    v[i] = q < G ? __ldcg(pc + q) : 0.0;
                }
#pragma unroll
                for (int i = 0; i < PQR_MAX_GRID / 8; ++i) t += v[i];
            }
            t += __shfl_xor_sync(0xffffffffu, t, 1);
            t += __shfl_xor_sync(0xffffffffu, t, 2);
            t += __shfl_xor_sync(0xffffffffu, t, 4);
            if (c < k && sub == 0) tot[c] = t;
        }
        __syncthreads();
    };

    int step = 0;  // barriers passed: selects the buffers
    dots(0, 0, S, false);
    if (r0 == 0)
        for (int c = threadIdx.x; c < k; c += blockDim.x) Ajg[c] = S[(size_t)c * ld];
    for (int j = 0; j < k; ++j, ++step) {
        if (!grid_barrier(count, gen, G, err, limit)) return;
        read_totals(j, step);
        const int par = step & 1;
        const double s2 = tot[j];
        const double xj = __ldcg(Ajg + (size_t)par * k + j);
        double bt = xj, inv = 0.0, tu = 0.0;
        if (s2 > 0.0) {
            const double sig = sqrt(s2);
            bt = xj >= 0.0 ? -sig : sig;
            inv = 1.0 / (xj - bt);  // |xj - bt| = |xj| + sig >= sig > 0
            tu = (bt - xj) / bt;
        }
        for (int c = j + 1 + threadIdx.x; c < k; c += blockDim.x)
            wv[c] = tu * (tot[c] - bt * __ldcg(Ajg + (size_t)par * k + c)) * inv;
        // column j becomes the reflector v (v_j = 1 implicit, beta on the diagonal)
        const int rl0 = max(0, j - r0);
        for (int rl = rl0 + threadIdx.x; rl < nrl; rl += blockDim.x)
            S[(size_t)j * ld + rl] = (r0 + rl == j) ? bt : S[(size_t)j * ld + rl] * inv;
        if (threadIdx.x == 0) {
            tau_s[j] = tu;
            beta_s[j] = bt;
        }
        __syncthreads();
        if (tu != 0.0) {
            const double* v = S + (size_t)j * ld;
            for (int c = j + 1 + warp; c < k; c += nw) {
                const double w = wv[c];
                double* a = S + (size_t)c * ld;
                for (int rl = rl0 + lane; rl < nrl; rl += 32) a[rl] = fma(-w, (r0 + rl == j) ? 1.0 : v[rl], a[rl]);
            }
        }
        __syncthreads();
        if (j + 1 < k) {
            dots(j + 1, (step + 1) & 1, S, false);
            if (j + 1 >= r0 && j + 1 < r1)
                for (int c = j + 1 + threadIdx.x; c < k; c += blockDim.x)
                    Ajg[(size_t)((step + 1) & 1) * k + c] = S[(size_t)c * ld + (j + 1 - r0)];
        }
    }

    // Q = H_0 ... H_{k-1} [I; 0], applied from the last reflector back
    int jn = k - 1;
    while (jn >= 0 && tau_s[jn] == 0.0) --jn;  // identical in every CTA
    if (jn >= 0) dots(jn, step & 1, Qs, true);
    while (jn >= 0) {
        const int j = jn;
        if (!grid_barrier(count, gen, G, err, limit)) return;
        read_totals(j, step);
        const double tu = tau_s[j];
        const int rl0 = max(0, j - r0);
        const double* v = S + (size_t)j * ld;
        for (int c = j + warp; c < k; c += nw) {
            const double w = tu * tot[c];
            double* q = Qs + (size_t)c * ld;
            for (int rl = rl0 + lane; rl < nrl; rl += 32) q[rl] = fma(-w, (r0 + rl == j) ? 1.0 : v[rl], q[rl]);
        }
        __syncthreads();
        ++step;
        jn = j - 1;
        while (jn >= 0 && tau_s[jn] == 0.0) --jn;
        if (jn >= 0) dots(jn, step & 1, Qs, true);
    }

    // signs so that diag(R) >= 0: column c of Q and row c of R times sgn(beta_c)
    for (int t = threadIdx.x; t < nrl * k; t += blockDim.x) {
        const int rl = t / k, c = t - rl * k;
        const double sg = beta_s[c] < 0.0 ? -1.0 : 1.0;
        Q[(size_t)(r0 + rl) * k + c] = sg * Qs[(size_t)c * ld + rl];
    }
    for (int t = threadIdx.x; t < nrl * k; t += blockDim.x) {
        const int rl = t / k, c = t - rl * k, jr = r0 + rl;
        if (jr >= k) continue;
        const double sg = beta_s[jr] < 0.0 ? -1.0 : 1.0;
        double v = 0.0;
        if (c == jr) v = fabs(beta_s[jr]);
        else if (c > jr) v = sg * S[(size_t)c * ld + rl];
        R[(size_t)jr * k + c] = v;
    }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi in a single launch: one thread-block cluster per matrix,
// its warps share the round's pairs; columns live in global memory and are
// read and written through L2 (ld.cg / st.cg); a cluster barrier (release /
// acquire) separates rounds.  Every thread runs every barrier, so the
// cluster cannot wait on a thread that left.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Per pair only the cross product g_p.g_q is formed: the squared column
// norms are tracked (a <- a - t c, b <- b + t c for the rotation with t =
// tan(theta)) and recomputed exactly at the start of every sweep; for k <=
// 256 the pair's columns stay in registers between the product and the
// rotation.
__global__ void __launch_bounds__(256) k_jacobi_cluster(double* __restrict__ Gt, double* __restrict__ Wt, int k,
                                                       int n, int max_sweeps, double tol,
                                                       unsigned long long* __restrict__ off,
                                                       double* __restrict__ nrm, int csize,
                                                       int* __restrict__ status) {
    constexpr int RK = 8;  // cached entries per lane: k <= 32 RK
    const int b = blockIdx.x / csize, rank = blockIdx.x % csize;
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    // pairs dealt CTA-first (warp w of CTA r takes pairs w csize + r + ...):
    // dealt warp-first the 72 pairs of k = 144 sat on 9 of the 16 SMs, whose
    // FP64 pipes then set every round's length
    const int gw = (threadIdx.x >> 5) * csize + rank, nw = csize * warps;
    double* g = Gt + (size_t)b * k * k;
    double* wm = Wt ? Wt + (size_t)b * k * k : nullptr;
    double* nb2 = nrm + (size_t)b * k;
    unsigned long long* offb = off + (size_t)b * max_sweeps;
    const bool cached = k <= 32 * RK;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        for (int c = gw; c < k; c += nw) {
            const double* gc = g + (size_t)c * k;
            double a = 0.0;
            for (int i = lane; i < k; i += 32) {
                const double x = __ldcg(gc + i);
                a = fma(x, x, a);
            }
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) __stcg(nb2 + c, a);
        }
        cluster_sync();
        for (int r = 0; r < n - 1; ++r) {
            for (int p = gw; p < n / 2; p += nw) {
                auto pos = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + r) % (n - 1); };
                int P = pos(p), Q = pos(n - 1 - p);
                if (P >= k || Q >= k) continue;
                if (P > Q) { const int t = P; P = Q; Q = t; }
                double* gp = g + (size_t)P * k;
                double* gq = g + (size_t)Q * k;
                double* wp = wm ? wm + (size_t)P * k : nullptr;
                double* wq = wm ? wm + (size_t)Q * k : nullptr;
                // every load of the pair is issued before the first use, so a
                // round costs one L2 round trip instead of one per 32 entries
                const double a = __ldcg(nb2 + P), bb = __ldcg(nb2 + Q);
                double xr[RK], yr[RK];
                double c = 0.0;
                if (cached) {
#pragma unroll
                    for (int u = 0; u < RK; ++u) {
                        const int i = lane + 32 * u;
                        xr[u] = i < k ? __ldcg(gp + i) : 0.0;
                        yr[u] = i < k ? __ldcg(gq + i) : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < RK; ++u) c = fma(xr[u], yr[u], c);
                } else {
                    for (int i = lane; i < k; i += 32) c = fma(__ldcg(gp + i), __ldcg(gq + i), c);
                }
                for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                if (a < 1e-280 || bb < 1e-280) continue;  // zero or near underflow: nothing to rotate
                const double rel = fabs(c) / (sqrt(a) * sqrt(bb));
                if (!(rel > tol)) continue;
                if (lane == 0) atomicMax(offb + sw, 1ull);  // this sweep rotated
                const double z = (bb - a) / (2.0 * c);
                const double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                if (cached) {
#pragma unroll
                    for (int u = 0; u < RK; ++u) {
                        const int i = lane + 32 * u;
                        if (i < k) {
                            __stcg(gp + i, cs * xr[u] - sn * yr[u]);
                            __stcg(gq + i, sn * xr[u] + cs * yr[u]);
                        }
                    }
                } else {
                    for (int i = lane; i < k; i += 32) {
                        const double x = __ldcg(gp + i), y = __ldcg(gq + i);
                        __stcg(gp + i, cs * x - sn * y);
                        __stcg(gq + i, sn * x + cs * y);
                    }
                }
                if (lane == 0) {
                    __stcg(nb2 + P, a - t * c);
                    __stcg(nb2 + Q, bb + t * c);
                }
                if (wm) {
                    if (cached) {
                        // all W loads of the pair in flight together
                        double ur[RK], vr[RK];
#pragma unroll
                        for (int u = 0; u < RK; ++u) {
                            const int i = lane + 32 * u;
                            ur[u] = i < k ? __ldcg(wp + i) : 0.0;
                            vr[u] = i < k ? __ldcg(wq + i) : 0.0;
                        }
#pragma unroll
                        for (int u = 0; u < RK; ++u) {
                            const int i = lane + 32 * u;
                            if (i < k) {
                                __stcg(wp + i, cs * ur[u] - sn * vr[u]);
                                __stcg(wq + i, sn * ur[u] + cs * vr[u]);
                            }
                        }
                    } else {
                        for (int i = lane; i < k; i += 32) {
                            const double x = __ldcg(wp + i), y = __ldcg(wq + i);
                            __stcg(wp + i, cs * x - sn * y);
                            __stcg(wq + i, sn * x + cs * y);
                        }
                    }
                }
            }
            cluster_sync();
        }
        const unsigned long long rotated = __ldcg(offb + sw);
        cluster_sync();  // everyone has read this sweep's value before anyone moves on
        if (!rotated) break;
        // the last sweep still rotated: report that the cap was hit
        if (sw == max_sweeps - 1 && rank == 0 && threadIdx.x == 0 && status) atomicExch(status, 1);
    }
}

// ---------------------------------------------------------------------------
// The same one-sided Jacobi with the matrix in the cluster's distributed
// shared memory: column c of G^T (and of W^T) lives in CTA c % csize, slot
// c / csize, with its squared norm beside it.  The warp that rotates a pair
// reads and writes both columns in their owners' shared memory, so a
// round's data never leaves the cluster and its release/acquire barrier
// orders shared-memory traffic only (through L2 every round had to wait for
// its global stores).  Rounds, pairs, tolerance and the per-sweep status
// are those of k_jacobi_cluster; G^T and W^T are copied in at the start and
// out at the end.  Every thread runs every barrier, and after the last
// barrier a CTA touches only its own shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_jacobi_dsmem(double* __restrict__ Gt, double* __restrict__ Wt, int k, int n,
                                                     int max_sweeps, double tol,
                                                     unsigned long long* __restrict__ off, int* __restrict__ status) {
    namespace cg = cooperative_groups;
    extern __shared__ double jsm[];
    cg::cluster_group cl = cg::this_cluster();
    const int csize = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int b = blockIdx.x / csize;
    const int slots = (k + csize - 1) / csize;
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    // pairs dealt CTA-first (warp w of CTA r takes pairs w csize + r + ...):
    // dealt warp-first the 72 pairs of k = 144 sat on 9 of the 16 SMs, whose
    // FP64 pipes then set every round's length
    const int gw = (threadIdx.x >> 5) * csize + rank, nw = csize * warps;
    double* gs = jsm;                               // [slots][k]
    double* ws = gs + (size_t)slots * k;            // [slots][k], when W is accumulated
    double* ns = ws + (size_t)slots * k;            // [slots] squared column norms
    double* g = Gt + (size_t)b * k * k;
    double* wm = Wt ? Wt + (size_t)b * k * k : nullptr;
    unsigned long long* offb = off + (size_t)b * max_sweeps;
    for (int t = threadIdx.x; t < slots * k; t += blockDim.x) {
        const int sl = t / k, i = t - sl * k, c = sl * csize + rank;
        gs[t] = c < k ? g[(size_t)c * k + i] : 0.0;
        if (wm) ws[t] = c < k ? wm[(size_t)c * k + i] : 0.0;
    }
    cluster_sync();
    auto gcol = [&](int c) { return cl.map_shared_rank(gs + (size_t)(c / csize) * k, c % csize); };
    auto wcol = [&](int c) { return cl.map_shared_rank(ws + (size_t)(c / csize) * k, c % csize); };
    auto ncol = [&](int c) { return cl.map_shared_rank(ns + c / csize, c % csize); };
    constexpr int RK = 8;  // cached entries per lane: k <= 32 RK
    const bool cached = k <= 32 * RK;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        // exact squared norms of the own columns at the start of every sweep
        for (int sl = threadIdx.x >> 5; sl < slots; sl += warps) {
            const double* x = gs + (size_t)sl * k;
            double a = 0.0;
            for (int i = lane; i < k; i += 32) a = fma(x[i], x[i], a);
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) ns[sl] = a;
        }
        cluster_sync();
        for (int r = 0; r < n - 1; ++r) {
            for (int p = gw; p < n / 2; p += nw) {
                auto pos = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + r) % (n - 1); };
                int P = pos(p), Q = pos(n - 1 - p);
                if (P >= k || Q >= k) continue;
                if (P > Q) { const int t = P; P = Q; Q = t; }
                double* gp = gcol(P);
                double* gq = gcol(Q);
                double* np = ncol(P);
                double* nq = ncol(Q);
                const double a = *np, bb = *nq;
                double xr[RK], yr[RK];
                double c = 0.0;
                if (cached) {
#pragma unroll
                    for (int u = 0; u < RK; ++u) {
                        const int i = lane + 32 * u;
                        xr[u] = i < k ? gp[i] : 0.0;
                        yr[u] = i < k ? gq[i] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < RK; ++u) c = fma(xr[u], yr[u], c);
                } else {
                    for (int i = lane; i < k; i += 32) c = fma(gp[i], gq[i], c);
                }
                for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                if (a < 1e-280 || bb < 1e-280) continue;  // zero or near underflow: nothing to rotate
                const double rel = fabs(c) / (sqrt(a) * sqrt(bb));
                if (!(rel > tol)) continue;
                if (lane == 0) atomicMax(offb + sw, 1ull);  // this sweep rotated
                const double z = (bb - a) / (2.0 * c);
                const double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                if (cached) {
#pragma unroll
                    for (int u = 0; u < RK; ++u) {
                        const int i = lane + 32 * u;
                        if (i < k) {
                            gp[i] = cs * xr[u] - sn * yr[u];
                            gq[i] = sn * xr[u] + cs * yr[u];
                        }
                    }
                } else {
                    for (int i = lane; i < k; i += 32) {
                        const double x = gp[i], y = gq[i];
                        gp[i] = cs * x - sn * y;
                        gq[i] = sn * x + cs * y;
                    }
                }
                if (lane == 0) {
                    *np = a - t * c;
                    *nq = bb + t * c;
                }
                if (wm) {
                    double* wp = wcol(P);
                    double* wq = wcol(Q);
                    for (int i = lane; i < k; i += 32) {
                        const double x = wp[i], y = wq[i];
                        wp[i] = cs * x - sn * y;
                        wq[i] = sn * x + cs * y;
                    }
                }
            }
            cluster_sync();
        }
        const unsigned long long rotated = __ldcg(offb + sw);
        cluster_sync();  // everyone has read this sweep's value before anyone moves on
        if (!rotated) break;
        if (sw == max_sweeps - 1 && rank == 0 && threadIdx.x == 0 && status) atomicExch(status, 1);
    }
    // own columns back to global memory
    for (int t = threadIdx.x; t < slots * k; t += blockDim.x) {
        const int sl = t / k, i = t - sl * k, c = sl * csize + rank;
        if (c < k) {
            g[(size_t)c * k + i] = gs[t];
            if (wm) wm[(size_t)c * k + i] = ws[t];
        }
    }
}

constexpr size_t JACOBI_DSMEM_MAX = 200 * 1024;
inline size_t jacobi_dsmem_bytes(int k, int csize) {
    const size_t slots = (size_t)(k + csize - 1) / csize;
    return sizeof(double) * (2 * slots * k + slots);
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
    if (a < 1e-280 || bb < 1e-280) return;  // zero or near underflow: nothing to rotate
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

// after the per-round fallback: the cap was hit when the last sweep rotated
__global__ void k_jacobi_status(const unsigned long long* __restrict__ off, int nb, int max_sweeps, double tol,
                                int* __restrict__ status) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (!(__longlong_as_double((long long)off[(size_t)(max_sweeps - 1) * nb + b]) < tol) &&
            off[(size_t)(max_sweeps - 1) * nb + b] != 0ull)
            atomicExch(status, 1);
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
// A pair counts as orthogonal at |g_p.g_q| <= tol |g_p||g_q|.  The computed
// cosine of two length-k columns carries rounding of about sqrt(k) 2^-53,
// so the bound follows k (4 sqrt(k) eps, the one-sided Jacobi criterion of
// LAPACK's dgesvj with a safety factor) and never goes below 1e-15.
inline double jacobi_tol(int k) { return std::max(1e-15, 4.0 * std::sqrt((double)k) * 0x1p-53); }

}  // namespace

// ---------------------------------------------------------------------------
size_t qr_ws_bytes(int N, int k) {
    const size_t nch = (size_t)(N + QR_CHUNK - 1) / QR_CHUNK;
    return sizeof(double) * (3 * (size_t)k * N + (size_t)k * k + 3 * (size_t)k + nch * k) + 256;
}

// Grid of the persistent QR on the current device (0: it does not apply --
// the panel slabs do not fit in shared memory or the device cannot run a
// cooperative launch), and its rows per CTA.
struct PqrPlan {
    int grid = 0, nr = 0;
    size_t smem = 0;
};
PqrPlan pqr_plan(int N, int k) {
    PqrPlan p;
    static std::mutex mu;
    static int nsm[64], coop[64];
    static unsigned long long known = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return p;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!(known >> dev & 1ull)) {
            if (cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm[dev] = 0;
            if (cudaDeviceGetAttribute(&coop[dev], cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) coop[dev] = 0;
            cudaGetLastError();
            known |= 1ull << dev;
        }
        if (!coop[dev] || nsm[dev] <= 0) return p;
        int g = std::min(std::min(nsm[dev], PQR_MAX_GRID), (N + PQR_MIN_ROWS - 1) / PQR_MIN_ROWS);
        if (g < 1) g = 1;
        const int nr = (N + g - 1) / g;
        const size_t smem = sizeof(double) * (2 * (size_t)k * (nr | 1) + 4 * (size_t)k);  // odd column stride
        if (smem > 200 * 1024) return p;
        p.grid = (N + nr - 1) / nr;
        p.nr = nr;
        p.smem = smem;
    }
    return p;
}

cudaError_t qr(const double* Y, int N, int k, double* Q, double* R, void* ws, cudaStream_t s, int* err) {
    if (N < k || k <= 0) return cudaErrorInvalidValue;
    const PqrPlan pp = pqr_plan(N, k);
    if (pp.grid > 0) {
        // ws: [err int | barrier count, generation] (256 B) | P [2][k][grid] | row j [2][k]
        char* w = (char*)ws;
        int* e_flag = err ? err : (int*)w;
        unsigned* bar = (unsigned*)(w + 16);
        double* P = (double*)(w + 256);
        double* Ajg = P + 2 * (size_t)pp.grid * k;
        // a caller's flag is not cleared here: it may hold an earlier time-out
        cudaError_t e = cudaMemsetAsync(w, 0, 256, s);
        if (e) return e;
        static std::mutex amu;
        static unsigned long long attr_done = 0;
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e) return e;
        {
            std::lock_guard<std::mutex> lock(amu);
            if (!(attr_done >> dev & 1ull)) {
                e = cudaFuncSetAttribute(k_qr_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                if (e) return e;
                attr_done |= 1ull << dev;
            }
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)pp.grid, 1, 1);
        cfg.blockDim = dim3(PQR_THREADS, 1, 1);
        cfg.dynamicSmemBytes = pp.smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        ++g_launches;
        return cudaLaunchKernelEx(&cfg, k_qr_persistent, Y, N, k, pp.nr, Q, R, P, Ajg, bar, e_flag,
                                  PQR_WAIT_CYCLES);
    }
    const int nch = (N + QR_CHUNK - 1) / QR_CHUNK;
    double* At = (double*)ws;
    double* V = At + (size_t)k * N;
    double* Qt = V + (size_t)k * N;
    double* Rtmp = Qt + (size_t)k * N;
    double* tau = Rtmp + (size_t)k * k;
    double* beta = tau + k;  // diagonal of R before the sign fix
    double* Aj = beta + k;
    double* P = Aj + k;
    const int dims[2] = {N, k}, perm[2] = {1, 0};
    cudaError_t e = permute(Y, At, 2, dims, perm, s);
    if (e) return e;
    e = cudaMemsetAsync(V, 0, sizeof(double) * (size_t)k * N, s);
    if (e) return e;
    for (int j = 0; j < k; ++j) {
        const dim3 grid(nch, k - j);
        ++g_launches;
        k_qr_dots<<<grid, QR2_THREADS, 0, s>>>(At, N, k, j, P, Aj);
        ++g_launches;
        k_qr_update<<<grid, QR2_THREADS, 0, s>>>(At, V, tau, beta, Rtmp, N, k, j, nch, P, Aj);
    }
    ++g_launches;
    k_eye_rows<<<grid_for((size_t)k * N), 256, 0, s>>>(Qt, N, k);
    for (int j = k - 1; j >= 0; --j) {
        const dim3 grid(nch, k - j);
        ++g_launches;
        k_qt_dots<<<grid, QR2_THREADS, 0, s>>>(Qt, V, tau, N, k, j, P);
        ++g_launches;
        k_qt_update<<<grid, QR2_THREADS, 0, s>>>(Qt, V, tau, N, k, j, nch, P);
    }
    ++g_launches;
    k_qr_out<<<grid_for((size_t)N * k), 256, 0, s>>>(Qt, beta, Rtmp, Q, R, N, k);
    return cudaGetLastError();
}

// Cluster size for the Jacobi kernel on the current device: 16 CTAs when the
// device accepts that non-portable size, else 8, else 0 (per-round launches).
// Decided once per device from occupancy queries, which launch nothing, so
// the first call may come inside a stream capture.
int jacobi_cluster_size() {
    static std::mutex mu;
    static int cached[64];
    static unsigned long long known = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (known >> dev & 1ull) return cached[dev];
    int cs = 0;
    if (cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    for (int want : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)want, 1, 1);
        cfg.blockDim = dim3(256, 1, 1);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = want;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_jacobi_cluster, &cfg) == cudaSuccess && nclusters > 0) {
            cs = want;
            break;
        }
        cudaGetLastError();
    }
    cached[dev] = cs;
    known |= 1ull << dev;
    return cs;
}

// Jacobi on nb matrices: one cluster per matrix when the device allows it,
// else one launch per round.  *status (optional) becomes 1 when a matrix
// still needed rotations in the last allowed sweep.
// Whether the shared-memory Jacobi can run with `bytes` of shared memory per
// CTA in a cluster of csize on the current device (attributes set once per
// device; occupancy queries launch nothing).
bool jacobi_dsmem_ok(size_t bytes, int csize) {
    static std::mutex mu;
    static unsigned long long attr_set = 0;
    if (bytes > JACOBI_DSMEM_MAX) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!(attr_set >> dev & 1ull)) {
            if (cudaFuncSetAttribute(k_jacobi_dsmem, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
                cudaFuncSetAttribute(k_jacobi_dsmem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)JACOBI_DSMEM_MAX) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            attr_set |= 1ull << dev;
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)csize, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_jacobi_dsmem, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters > 0;
}

cudaError_t jacobi(double* Gt, double* Wt, int k, int n, int nb, unsigned long long* off, double* nrm,
                   int* status, cudaStream_t s) {
    const int csize = jacobi_cluster_size();
    if (csize > 0) {
        const size_t dsm = jacobi_dsmem_bytes(k, csize);
        const bool in_smem = jacobi_dsmem_ok(dsm, csize);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nb * csize), 1, 1);
        cfg.blockDim = dim3(256, 1, 1);
        cfg.dynamicSmemBytes = in_smem ? dsm : 0;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = csize;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        ++g_launches;
        if (in_smem)
            return cudaLaunchKernelEx(&cfg, k_jacobi_dsmem, Gt, Wt, k, n, JACOBI_MAX_SWEEPS, jacobi_tol(k), off,
                                      status);
        return cudaLaunchKernelEx(&cfg, k_jacobi_cluster, Gt, Wt, k, n, JACOBI_MAX_SWEEPS, jacobi_tol(k), off, nrm,
                                  csize, status);
    }
    for (int sw = 0; sw < JACOBI_MAX_SWEEPS; ++sw)
        for (int r = 0; r < n - 1; ++r) {
            ++g_launches;
            k_jacobi_round<<<dim3(n / 2, nb), 32, 0, s>>>(Gt, Wt, k, n, r, sw, off, jacobi_tol(k));
        }
    if (status) {
        ++g_launches;
        k_jacobi_status<<<1, 256, 0, s>>>(off, nb, JACOBI_MAX_SWEEPS, jacobi_tol(k), status);
    }
    return cudaGetLastError();
}

// scratch: status word (256 bytes), G^T and W^T (k x k each), squared column
// norms (k), per-sweep words (the cluster kernels' "rotated" flags, the
// per-round kernels' off-diagonal maxima)
constexpr size_t svd_ws_bytes_c(int k) {
    return 256 + sizeof(double) * (2 * (size_t)k * k + k) + sizeof(unsigned long long) * JACOBI_MAX_SWEEPS + 256;
}
size_t svd_ws_bytes(int k) { return svd_ws_bytes_c(k); }

cudaError_t svd(const double* G, int k, double* U, double* S, double* V, void* ws, cudaStream_t s, int* status) {
    if (k <= 0 || k > 1024) return cudaErrorInvalidValue;
    int* st = (int*)ws;  // 1 if the Jacobi sweep cap was hit
    double* Gt = (double*)((char*)ws + 256);
    double* Wt = Gt + (size_t)k * k;
    double* nrm = Wt + (size_t)k * k;
    unsigned long long* off = (unsigned long long*)(nrm + k);
    cudaError_t e = cudaMemsetAsync(off, 0, sizeof(unsigned long long) * JACOBI_MAX_SWEEPS, s);
    if (e) return e;
    e = cudaMemsetAsync(st, 0, sizeof(int), s);
    if (e) return e;
    ++g_launches;
    k_transpose_batch<<<grid_for((size_t)k * k), 256, 0, s>>>(G, Gt, k, 1);
    ++g_launches;
    k_eye_batch<<<grid_for((size_t)k * k), 256, 0, s>>>(Wt, k, 1);
    const int n = k + (k & 1);
    e = jacobi(Gt, Wt, k, n, 1, off, nrm, status ? status : st, s);
    if (e) return e;
    ++g_launches;
    k_jacobi_finish<<<1, 256, sizeof(double) * k, s>>>(Gt, Wt, k, U, S, V);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Eigenvalues of a small real m x m matrix (m <= SMALL_EIG_MAX): reduction to
// upper Hessenberg form by Householder reflections, then the QR algorithm in
// complex arithmetic with one Wilkinson shift per step (the eigenvalue of
// the trailing 2 x 2 block nearer its last diagonal entry; an exceptional
// shift after 10 and 20 steps without deflation) and deflation where a
// subdiagonal entry falls below 2^-52 of its two diagonal neighbours.  Only
// the active diagonal block is updated: the eigenvalues of a block upper
// triangular matrix are those of its diagonal blocks.  One thread; the
// matrix lives in shared memory.
// ---------------------------------------------------------------------------
namespace {
struct cd {
    double re, im;
};
__device__ __forceinline__ cd c_mk(double r, double i) { return cd{r, i}; }
__device__ __forceinline__ cd c_add(cd a, cd b) { return c_mk(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cd c_sub(cd a, cd b) { return c_mk(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cd c_mul(cd a, cd b) { return c_mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
__device__ __forceinline__ cd c_conj(cd a) { return c_mk(a.re, -a.im); }
__device__ __forceinline__ cd c_scale(cd a, double t) { return c_mk(a.re * t, a.im * t); }
__device__ __forceinline__ double c_abs(cd a) { return hypot(a.re, a.im); }
__device__ __forceinline__ double c_l1(cd a) { return fabs(a.re) + fabs(a.im); }
// a / b by Smith's scaling, which avoids overflow in |b|^2
__device__ __forceinline__ cd c_div(cd a, cd b) {
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, den = b.re + b.im * r;
        return c_mk((a.re + a.im * r) / den, (a.im - a.re * r) / den);
    }
    const double r = b.re / b.im, den = b.im + b.re * r;
    return c_mk((a.re * r + a.im) / den, (a.im * r - a.re) / den);
}
// principal square root
__device__ __forceinline__ cd c_sqrt(cd z) {
    const double r = c_abs(z);
    if (r == 0.0) return c_mk(0.0, 0.0);
    const double t = sqrt(0.5 * (r + fabs(z.re)));
    if (z.re >= 0.0) return c_mk(t, z.im / (2.0 * t));
    return c_mk(fabs(z.im) / (2.0 * t), z.im >= 0.0 ? t : -t);
}

constexpr int SMALL_EIG_MAX = 32;

__global__ void k_small_eig(const double* __restrict__ H, int m, int ldh, double period, double* __restrict__ out,
                            int* __restrict__ status, double* __restrict__ evout) {
    __shared__ double R[SMALL_EIG_MAX][SMALL_EIG_MAX];
    __shared__ cd Z[SMALL_EIG_MAX][SMALL_EIG_MAX];
    __shared__ cd ev[SMALL_EIG_MAX];
    __shared__ double v[SMALL_EIG_MAX];
    __shared__ double gc[SMALL_EIG_MAX];
    __shared__ cd gs[SMALL_EIG_MAX];
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double hn = 0.0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            R[i][j] = H[(size_t)i * ldh + j];
            hn = fmax(hn, fabs(R[i][j]));
        }
    // Householder: R <- P R P with P = I - 2 v v^T / |v|^2 zeroing column k below k+1
    for (int k = 0; k + 2 < m; ++k) {
        double a2 = 0.0;
        for (int i = k + 1; i < m; ++i) a2 += R[i][k] * R[i][k];
        if (a2 == 0.0) continue;
        const double alpha = R[k + 1][k] > 0.0 ? -sqrt(a2) : sqrt(a2);
        double vn2 = 0.0;
        for (int i = k + 1; i < m; ++i) {
            v[i] = R[i][k] - (i == k + 1 ? alpha : 0.0);
            vn2 += v[i] * v[i];
        }
        if (vn2 == 0.0) continue;
        for (int j = k; j < m; ++j) {
            double t = 0.0;
            for (int i = k + 1; i < m; ++i) t += v[i] * R[i][j];
            t *= 2.0 / vn2;
            for (int i = k + 1; i < m; ++i) R[i][j] -= t * v[i];
        }
        for (int i = 0; i < m; ++i) {
            double t = 0.0;
            for (int j = k + 1; j < m; ++j) t += R[i][j] * v[j];
            t *= 2.0 / vn2;
            for (int j = k + 1; j < m; ++j) R[i][j] -= t * v[j];
        }
        for (int i = k + 2; i < m; ++i) R[i][k] = 0.0;
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Z[i][j] = c_mk(R[i][j], 0.0);
    const double eps = 0x1p-52;
    const double tiny = hn > 0.0 ? eps * hn * 1e-30 : 1e-300;
    int st = 0, hi = m - 1, its = 0, total = 0;
    while (hi >= 0) {
        if (hi == 0) {
            ev[0] = Z[0][0];
            break;
        }
        int l = hi;
        for (; l > 0; --l) {
            const double sc = c_l1(Z[l - 1][l - 1]) + c_l1(Z[l][l]);
            if (c_l1(Z[l][l - 1]) <= eps * sc || c_l1(Z[l][l - 1]) <= tiny) {
                Z[l][l - 1] = c_mk(0.0, 0.0);
                break;
            }
        }
        if (l == hi) {
            ev[hi] = Z[hi][hi];
            --hi;
            its = 0;
            continue;
        }
        if (++total > 60 * m) {
            st = 1;  // not converged: report the current diagonal
            for (int i = 0; i <= hi; ++i) ev[i] = Z[i][i];
            break;
        }
        cd shift;
        if (its == 10 || its == 20) {
            shift = c_add(Z[hi][hi], c_mk(0.75 * c_abs(Z[hi][hi - 1]), 0.0));
        } else {
            const cd a = Z[hi - 1][hi - 1], b = Z[hi - 1][hi], c = Z[hi][hi - 1], d = Z[hi][hi];
            const cd half = c_scale(c_add(a, d), 0.5), dif = c_scale(c_sub(a, d), 0.5);
            const cd disc = c_sqrt(c_add(c_mul(dif, dif), c_mul(b, c)));
            const cd mu1 = c_add(half, disc), mu2 = c_sub(half, disc);
            shift = c_abs(c_sub(mu1, d)) <= c_abs(c_sub(mu2, d)) ? mu1 : mu2;
        }
        ++its;
        for (int i = l; i <= hi; ++i) Z[i][i] = c_sub(Z[i][i], shift);
        // Z - shift = Q R by Givens rotations G_k on rows k, k+1 ...
        for (int k = l; k < hi; ++k) {
            const cd f = Z[k][k], g = Z[k + 1][k];
            const double fa = c_abs(f), ga = c_abs(g);
            double c;
            cd sn;
            if (ga == 0.0) {
                c = 1.0;
                sn = c_mk(0.0, 0.0);
            } else if (fa == 0.0) {
                c = 0.0;
                sn = c_scale(c_conj(g), 1.0 / ga);
            } else {
                const double r = hypot(fa, ga);
                c = fa / r;
                sn = c_scale(c_mul(c_scale(f, 1.0 / fa), c_conj(g)), 1.0 / r);
            }
            gc[k] = c;
            gs[k] = sn;
            for (int j = k; j <= hi; ++j) {
                const cd x = Z[k][j], y = Z[k + 1][j];
                Z[k][j] = c_add(c_scale(x, c), c_mul(sn, y));
                Z[k + 1][j] = c_sub(c_scale(y, c), c_mul(c_conj(sn), x));
            }
        }
        // ... then R Q: G_k^H on columns k, k+1
        for (int k = l; k < hi; ++k) {
            const double c = gc[k];
            const cd sn = gs[k];
            const int last = min(k + 2, hi);
            for (int i = l; i <= last; ++i) {
                const cd x = Z[i][k], y = Z[i][k + 1];
                Z[i][k] = c_add(c_scale(x, c), c_mul(y, c_conj(sn)));
                Z[i][k + 1] = c_sub(c_scale(y, c), c_mul(x, sn));
            }
        }
        for (int i = l; i <= hi; ++i) Z[i][i] = c_add(Z[i][i], shift);
    }
    // descending modulus (stable insertion sort)
    for (int i = 1; i < m; ++i) {
        const cd x = ev[i];
        const double ax = c_abs(x);
        int j = i - 1;
        while (j >= 0 && c_abs(ev[j]) < ax) {
            ev[j + 1] = ev[j];
            --j;
        }
        ev[j + 1] = x;
    }
    const double a0 = c_abs(ev[0]);
    if (a0 == 0.0) st = st ? st : 2;
    for (int i = 0; i < m; ++i) {
        const double ai = c_abs(ev[i]);
        const cd r = a0 > 0.0 ? c_div(ev[i], ev[0]) : c_mk(0.0, 0.0);
        out[i] = r.re;
        out[m + i] = r.im;
        out[2 * m + i] = ai;
        out[3 * m + i] = (a0 > 0.0 && ai > 0.0) ? -log(ai / a0) / period : INFINITY;
        if (evout) {
            evout[2 * i] = ev[i].re;
            evout[2 * i + 1] = ev[i].im;
        }
    }
    if (status) *status = st;
}

// Ritz vectors of the leading eigenvalues by inverse iteration on the small
// matrix: (H - mu I) y = y_prev with mu = lambda (1 + 1e-10), three solves
// after one LU factorisation with partial pivoting (complex), y normalised.
// A real eigenvalue gives Re y; a complex pair gives Re y and Im y (the
// conjugate's eigenvector adds nothing real).  One thread.
__global__ void k_ritz_basis(const double* __restrict__ H, int m, int ldh, const double* __restrict__ ev, int nvec,
                             double* __restrict__ Y) {
    __shared__ cd L[SMALL_EIG_MAX][SMALL_EIG_MAX];
    __shared__ cd y[SMALL_EIG_MAX];
    __shared__ int piv[SMALL_EIG_MAX];
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double scale = hypot(ev[0], ev[1]);
    const double tiny = (scale > 0.0 ? scale : 1.0) * 1e-300;
    int out = 0;
    for (int i = 0; i < m && out < nvec; ++i) {
        const cd lam = c_mk(ev[2 * i], ev[2 * i + 1]);
        const cd mu = c_add(lam, c_scale(lam, 1e-10));
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c) L[r][c] = c_mk(H[(size_t)r * ldh + c] - (r == c ? mu.re : 0.0), r == c ? -mu.im : 0.0);
        // LU with partial pivoting, in place
        for (int c = 0; c < m; ++c) {
            int p = c;
            double best = c_abs(L[c][c]);
            for (int r = c + 1; r < m; ++r)
                if (c_abs(L[r][c]) > best) { best = c_abs(L[r][c]); p = r; }
            piv[c] = p;
            if (p != c)
                for (int q = 0; q < m; ++q) { const cd t = L[c][q]; L[c][q] = L[p][q]; L[p][q] = t; }
            if (c_abs(L[c][c]) < tiny) L[c][c] = c_mk(tiny, 0.0);
            for (int r = c + 1; r < m; ++r) {
                const cd f = c_div(L[r][c], L[c][c]);
                L[r][c] = f;
                for (int q = c + 1; q < m; ++q) L[r][q] = c_sub(L[r][q], c_mul(f, L[c][q]));
            }
        }
        for (int r = 0; r < m; ++r) y[r] = c_mk(1.0, 0.0);
        for (int it = 0; it < 3; ++it) {
            for (int c = 0; c < m; ++c)  // row interchanges, then L (unit lower) forward
                if (piv[c] != c) { const cd t = y[c]; y[c] = y[piv[c]]; y[piv[c]] = t; }
            for (int r = 0; r < m; ++r)
                for (int c = 0; c < r; ++c) y[r] = c_sub(y[r], c_mul(L[r][c], y[c]));
            for (int r = m - 1; r >= 0; --r) {  // U backward
                for (int c = r + 1; c < m; ++c) y[r] = c_sub(y[r], c_mul(L[r][c], y[c]));
                y[r] = c_div(y[r], L[r][r]);
            }
            double nrm = 0.0;
            for (int r = 0; r < m; ++r) nrm = hypot(nrm, c_abs(y[r]));
            const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
            for (int r = 0; r < m; ++r) y[r] = c_scale(y[r], inv);
        }
        for (int r = 0; r < m; ++r) Y[(size_t)out * m + r] = y[r].re;
        ++out;
        const bool pair = fabs(lam.im) > 1e-12 * (scale > 0.0 ? scale : 1.0);
        if (pair) {
            if (out < nvec) {
                for (int r = 0; r < m; ++r) Y[(size_t)out * m + r] = y[r].im;
                ++out;
            }
            if (i + 1 < m && fabs(ev[2 * (i + 1)] - lam.re) <= 1e-9 * scale &&
                fabs(ev[2 * (i + 1) + 1] + lam.im) <= 1e-9 * scale)
                ++i;  // skip the conjugate
        }
    }
    for (; out < nvec; ++out)  // fewer eigenvalues than vectors asked for
        for (int r = 0; r < m; ++r) Y[(size_t)out * m + r] = (r == out) ? 1.0 : 0.0;
}
}  // namespace

int small_eig_max() { return SMALL_EIG_MAX; }

cudaError_t small_eig(const double* H, int m, int ldh, double period, double* out, int* status, cudaStream_t s,
                      double* ev) {
    if (m < 1 || m > SMALL_EIG_MAX || ldh < m || !H || !out || !(period > 0.0)) return cudaErrorInvalidValue;
    ++g_launches;
    k_small_eig<<<1, 32, 0, s>>>(H, m, ldh, period, out, status, ev);
    return cudaGetLastError();
}

cudaError_t ritz_basis(const double* H, int m, int ldh, const double* ev, int nvec, double* Y, cudaStream_t s) {
    if (m < 1 || m > SMALL_EIG_MAX || ldh < m || nvec < 1 || nvec > m || !H || !ev || !Y) return cudaErrorInvalidValue;
    ++g_launches;
    k_ritz_basis<<<1, 32, 0, s>>>(H, m, ldh, ev, nvec, Y);
    return cudaGetLastError();
}

// Two independent SVDs in one Jacobi launch (two clusters); the layout of
// svd() per matrix: status word, then G^T, W^T, norms, per-sweep words
size_t svd2_ws_bytes(int k) {
    return 256 + sizeof(double) * 2 * (2 * (size_t)k * k + k) + sizeof(unsigned long long) * 2 * JACOBI_MAX_SWEEPS +
           256;
}

cudaError_t svd2(const double* G0, const double* G1, int k, double* U0, double* S0, double* V0, double* U1,
                 double* S1, double* V1, void* ws, cudaStream_t s, int* status) {
    if (k <= 0 || k > 1024) return cudaErrorInvalidValue;
    int* st = (int*)ws;
    double* Gt = (double*)((char*)ws + 256);        // [2][k][k]
    double* Wt = Gt + 2 * (size_t)k * k;             // [2][k][k]
    double* nrm = Wt + 2 * (size_t)k * k;            // [2][k]
    unsigned long long* off = (unsigned long long*)(nrm + 2 * (size_t)k);  // [2][sweeps]
    cudaError_t e = cudaMemsetAsync(off, 0, sizeof(unsigned long long) * 2 * JACOBI_MAX_SWEEPS, s);
    if (e) return e;
    e = cudaMemsetAsync(st, 0, sizeof(int), s);
    if (e) return e;
    ++g_launches;
    k_transpose_batch<<<grid_for((size_t)k * k), 256, 0, s>>>(G0, Gt, k, 1);
    ++g_launches;
    k_transpose_batch<<<grid_for((size_t)k * k), 256, 0, s>>>(G1, Gt + (size_t)k * k, k, 1);
    ++g_launches;
    k_eye_batch<<<grid_for(2 * (size_t)k * k), 256, 0, s>>>(Wt, k, 2);
    const int n = k + (k & 1);
    e = jacobi(Gt, Wt, k, n, 2, off, nrm, status ? status : st, s);
    if (e) return e;
    ++g_launches;
    k_jacobi_finish<<<1, 256, sizeof(double) * k, s>>>(Gt, Wt, k, U0, S0, V0);
    ++g_launches;
    k_jacobi_finish<<<1, 256, sizeof(double) * k, s>>>(Gt + (size_t)k * k, Wt + (size_t)k * k, k, U1, S1, V1);
    return cudaGetLastError();
}

size_t svals_ws_bytes(int k, int nb) {
    return sizeof(double) * (size_t)nb * ((size_t)k * k + k) + sizeof(unsigned long long) * JACOBI_MAX_SWEEPS * nb +
           256;
}

cudaError_t svals_normalised(const double* Gs, int k, int nb, double* out, void* ws, cudaStream_t s) {
    if (k <= 0 || k > 1024 || nb <= 0 || nb > 65535) return cudaErrorInvalidValue;
    double* Gt = (double*)ws;
    double* nrm = Gt + (size_t)nb * k * k;
    unsigned long long* off = (unsigned long long*)(nrm + (size_t)nb * k);
    cudaError_t e = cudaMemsetAsync(off, 0, sizeof(unsigned long long) * JACOBI_MAX_SWEEPS * nb, s);
    if (e) return e;
    ++g_launches;
    k_transpose_batch<<<grid_for((size_t)nb * k * k), 256, 0, s>>>(Gs, Gt, k, nb);
    const int n = k + (k & 1);
    e = jacobi(Gt, nullptr, k, n, nb, off, nrm, nullptr, s);
    if (e) return e;
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
constexpr size_t SVD_NOALLOC_BYTES = svd_ws_bytes_c(SVD_NOALLOC_MAX_K);
static __device__ __align__(256) unsigned char g_svd_scratch[SVD_NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};
}  // namespace

int svd_noalloc_max_k() { return SVD_NOALLOC_MAX_K; }

cudaError_t svd_noalloc(const double* G, int k, double* U, double* S, double* V, cudaStream_t s) {
    if (k <= 0 || k > SVD_NOALLOC_MAX_K) return cudaErrorInvalidValue;
    // every k accepted here needs at most the workspace of the largest k
    static_assert(svd_ws_bytes_c(SVD_NOALLOC_MAX_K) <= sizeof(g_svd_scratch),
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
    return svd(G, k, U, S, V, ws, s, nullptr);
}

}  // namespace ctm
