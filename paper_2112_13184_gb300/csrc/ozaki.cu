// Emulated-FP64 GEMM on the GB300 tensor cores (tcgen05 + TMEM + TMA).
//
// Each FP64 operand row (of A) or column (of B) is scaled by a power of two
// 2^e with max|x| <= 2^e and cut into s signed 8-bit digits,
//     x = 2^(e-8) * sum_t a_t 2^(-8t),   a_0 in [-256,256], a_t in [-128,127],
// computed with integer operations on the FP64 bit pattern (the FP64 pipe of
// GB300 is slow).  The scaled digits at_t = a_t 2^(-8t) are exact in BF16.
// C = A B is then the sum of BF16 slice products at_t * bt_u, accumulated
// on the tensor cores in FP32 over K-chunks of 256 and read out of TMEM
// after every chunk:
//   level 0 (t+u = 0) and level 1 (t+u = 1) are integer-valued (in units of
//   1 and 2^-8); over one chunk they stay below 2^24 units and are exact,
//   and are added to int32 registers;
//   all pairs with 2 <= t+u <= s-1 carry a weight <= 2^-16 and share one
//   FP32 accumulator, restarted every chunk so that the tensor cores'
//   rounding does not grow with the magnitude accumulated over K; the chunk
//   values are added in an FP32 register;
//   pairs with t+u >= s are dropped (same order as the slicing error).
// The result is assembled exactly in int64, C = 2^(eA+eB-16) (S0 + 2^-8 S1
// + F).  Error: the slicing, 2^(2-8s) max|row| max|col| K, plus the tensor
// cores' FP32 rounding of the levels >= 2 within a chunk, measured at about
// 2^-36 max|row| max|col| K; so 5 slices reach ~1e-11 relative per unit K
// and a 6th adds nothing.  Split-BF16 accumulated in FP32 over all of K
// cannot go below ~2^-24.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace ctm {
namespace oz {

constexpr int BM = 128;          // rows per CTA (one TMEM lane per row)
constexpr int BK = 32;           // K per pipeline stage (64 bytes: one SW64 row)
constexpr int CHUNK_KB = 8;      // k-blocks per exact chunk (K = 256)
constexpr int EPI_WARPS = 12;    // 3 warps per TMEM lane quarter
constexpr int THREADS = (EPI_WARPS + 2) * 32;  // + producer warp + MMA warp
constexpr int MAX_S = 6;

// A strided multi-index view: index i = (i_0, ..., i_{n-1}) in row-major
// order over dims, offset = sum_a i_a * stride[a].  Used to read operands as
// permuted views of larger tensors and to write results into permuted
// layouts, so that no FP64 permutation pass is needed.
struct View {
    int n;
    int dim[4];
    long long stride[4];
};
__host__ __device__ __forceinline__ long long view_offset(const View& v, long long i) {
    long long off = 0;
#pragma unroll
    for (int a = 3; a >= 0; --a) {
        if (a < v.n) {
            const long long q = i / v.dim[a];
            off += (i - q * v.dim[a]) * v.stride[a];
            i = q;
        }
    }
    return off;
}

// 32-bit decomposition (all view extents here are below 2^31)
__device__ __forceinline__ long long view_offset32(const View& v, unsigned i) {
    long long off = 0;
#pragma unroll
    for (int a = 3; a >= 0; --a) {
        if (a < v.n) {
            const unsigned dm = (unsigned)v.dim[a];
            const unsigned q = i / dm;
            off += (long long)(i - q * dm) * v.stride[a];
            i = q;
        }
    }
    return off;
}

// walks a view's indices in order, one add per step (carry on wrap)
struct Odometer {
    int idx[4];
    long long off;
    __device__ __forceinline__ void init(const View& v, unsigned i) {
        off = 0;
#pragma unroll
        for (int a = 3; a >= 0; --a) {
            idx[a] = 0;
            if (a < v.n) {
                const unsigned dm = (unsigned)v.dim[a];
                const unsigned q = i / dm;
                idx[a] = (int)(i - q * dm);
                off += (long long)idx[a] * v.stride[a];
                i = q;
            }
        }
    }
    __device__ __forceinline__ void step(const View& v) {
#pragma unroll
        for (int a = 3; a >= 0; --a) {
            if (a < v.n) {
                off += v.stride[a];
                if (++idx[a] < v.dim[a]) return;
                off -= (long long)v.dim[a] * v.stride[a];
                idx[a] = 0;
            }
        }
    }
};

// v * 2^k for finite v, through the exponent field when the result stays
// normal (the common case), else by ldexp
__device__ __forceinline__ double scale_pow2(double v, int k) {
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (v == 0.0) return v;
    if (e > 0 && e + k > 0 && e + k < 2047) return __longlong_as_double(b + ((long long)k << 52));
    return ldexp(v, k);
}

// Z * 2^E outside the normal FP64 range (rare): kept out of line so that its
// FP64 conversion and scaling are not if-converted into every element
__device__ __noinline__ double i64_ldexp_slow(long long Z, int E) {
    return ldexp((double)Z, E);
}

// Z * 2^E as an FP64 number (round to nearest even) with integer operations
// only: GB300's FP64 pipe is too slow to spend on every output element.
__device__ __forceinline__ double i64_ldexp(long long Z, int E) {
    if (Z == 0) return 0.0;
    const unsigned long long neg = Z < 0 ? 1ull : 0ull;
    unsigned long long m = neg ? (0ull - (unsigned long long)Z) : (unsigned long long)Z;
    int sh = (64 - __clzll((long long)m)) - 53;  // bits beyond a 53-bit mantissa
    unsigned long long mant;
    if (sh > 0) {
        const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        mant = m >> sh;
        if (rem > half || (rem == half && (mant & 1ull))) {
            ++mant;
            if (mant >> 53) {
                mant >>= 1;
                ++sh;
            }
        }
    } else {
        mant = m << (-sh);
    }
    const int be = E + sh + 52 + 1023;  // value = mant 2^(E+sh), mant in [2^52, 2^53)
    if (be <= 0 || be >= 2047) return i64_ldexp_slow(Z, E);  // outside the normal range
    return __longlong_as_double((long long)((neg << 63) | ((unsigned long long)be << 52) | (mant & ((1ull << 52) - 1))));
}

// round(f * 2^k) as int64 from the FP32 bit pattern (|f 2^k| < 2^62)
__device__ __forceinline__ long long f32_fixed(float f, int k) {
    const unsigned b = __float_as_uint(f);
    const int ex = (int)((b >> 23) & 0xff);
    if (ex == 0) return 0;  // zero or FP32 denormal: far below the resolution kept
    const long long mant = (long long)((b & 0x7fffff) | 0x800000);
    const int sh = ex - 150 + k;  // f 2^k = mant 2^sh
    long long v;
    if (sh >= 0) v = mant << sh;
    else if (sh <= -25) v = 0;
    else v = (mant + (1ll << (-sh - 1))) >> (-sh);
    return (b >> 31) ? -v : v;
}

// C = 2^(eA+eB-16) (S0 + S1/256 + F).  With T = 256 S0 + S1 (exact; |T| <
// 2^39 for K <= 16384 per split) and F kept to 2^-28 of an S0 unit (below
// 2^-44 of max|row| max|col|), Z = 2^20 T + round(2^28 F) is an exact int64
// and C = Z 2^(eA+eB-44).  escale = eA + eB - 16.  round(2^28 F) is taken
// from F's bit pattern: an FP32 -> int64 conversion instruction issues on
// the FP64 pipe, which GB300 runs at 2 lanes per clock per SM.
__device__ __forceinline__ double assemble(int S0, int S1, float F, int escale) {
    const long long T = (long long)S0 * 256 + (long long)S1;
    const long long Z = T * (1ll << 20) + f32_fixed(F, 28);  // F 2^28 < 2^62
    return i64_ldexp(Z, escale - 28);
}

__device__ __noinline__ double f32_ldexp_slow(float f, int E) { return ldexp((double)f, E); }

// f 2^E as an FP64 number for an FP32 f (the accumulator of the FP32-
// accumulated modes), built from the bit pattern: the exponent is rebiased
// and the 23-bit significand widened, integer instructions only.
__device__ __forceinline__ double f32_scaled(float f, int E) {
    const unsigned b = __float_as_uint(f);
    const int ex = (int)((b >> 23) & 0xff);
    if (ex == 0) return 0.0;                                      // zero or FP32 denormal
    if (ex == 255) return __longlong_as_double(0x7ff8000000000000ll);  // Inf/NaN accumulator
    const int be = ex - 127 + 1023 + E;
    if (be <= 0 || be >= 2047) return f32_ldexp_slow(f, E);       // outside the normal FP64 range
    return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                            ((unsigned long long)be << 52) |
                                            ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// ---------------------------------------------------------------------------
// slicing
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}
// row_exponent of the bit pattern of max|x| (integer operations only)
__device__ __forceinline__ int row_exponent_bits(unsigned long long mb) {
    if ((mb & 0x7fffffffffffffffull) == 0) return 0;
    const int E = (int)((mb >> 52) & 0x7ff);
    return E == 0 ? -1022 : E - 1022;
}
// exponent e with max|x| < 2^e (0 for an all-zero row; 1025 when the row
// holds an infinity or a NaN, which the products turn into NaN outputs)
__device__ __forceinline__ int row_exponent(double mx) {
    if (mx == 0.0) return 0;
    const int E = (int)((__double_as_longlong(mx) >> 52) & 0x7ff);
    return E == 0 ? -1022 : E - 1022;
}

// signed base-256 digits of round(x * 2^(8s - e)); |x| <= 2^e.  d[1..s-1]
// lie in [-128, 127] (Y = 256 Y' + d with Y' = floor((Y + 128) / 256)), d[0]
// carries the sign and the top.  Every index of d is static (unrolled over
// MAX_S), so d stays in registers.
__device__ __forceinline__ void digits_bits(unsigned long long b, int e, int s, int* d);
__device__ __forceinline__ void digits(double x, int e, int s, int* d) {
    digits_bits((unsigned long long)__double_as_longlong(x), e, s, d);
}
// the same from the FP64 bit pattern b
__device__ __forceinline__ void digits_bits(unsigned long long b, int e, int s, int* d) {
    int ex = (int)((b >> 52) & 0x7ff);
    unsigned long long mant = b & ((1ull << 52) - 1);
    if (ex == 0) ex = 1;
    else mant |= 1ull << 52;
    const int shift = ex - 1075 + 8 * s - e;  // x = mant 2^(ex-1075)
    long long Y;
    if (mant == 0) Y = 0;
    else if (shift >= 0) Y = (long long)(mant << shift);  // <= 2^(8s) by |x| <= 2^e
    else {
        const int sh = -shift;
        Y = sh >= 54 ? 0 : (long long)((mant + (1ull << (sh - 1))) >> sh);
    }
    if (b >> 63) Y = -Y;
#pragma unroll
    for (int t = MAX_S - 1; t >= 1; --t) {
        if (t < s) {
            const long long Yn = (Y + 128) >> 8;
            d[t] = (int)((uint32_t)Y - ((uint32_t)Yn << 8));  // Y - 256 Y', in [-128, 127]
            Y = Yn;
        } else {
            d[t] = 0;
        }
    }
    d[0] = (int)Y;
}

// A small int as an FP32 without a conversion instruction: 1.5 2^23 + d has
// the bit pattern 0x4B400000 + d for |d| < 2^22, so one FP32 subtraction
// recovers d exactly.
__device__ __forceinline__ float small_int_f32(int d) {
    return __int_as_float(0x4B400000 + d) - 12582912.0f;
}

// digit * 2^(-8t): at most 9 significant bits, exact in FP32 and BF16; the
// power of two is built from its exponent field
__device__ __forceinline__ __nv_bfloat16 slice_value(int digit, int t) {
    return __float2bfloat16_rn(small_int_f32(digit) * __int_as_float((127 - 8 * t) << 23));
}

// Consecutive k contiguous (innermost K stride 1): one warp per row.
__global__ void k_split_rows(const double* __restrict__ X, int R, int K, int K8, View rv, View kv, int s,
                             __nv_bfloat16* __restrict__ out, int* __restrict__ ex) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= R) return;
    const double* xr = X + view_offset32(rv, (unsigned)warp);
    auto at = [&](int k) { return xr[kv.n == 1 ? (long long)k * kv.stride[0] : view_offset32(kv, (unsigned)k)]; };
    // max |x| on the bit patterns: non-negative doubles order like integers,
    // and the integer pipe is far faster than GB300's FP64 pipe
    unsigned long long mb = 0;
    for (int k = lane; k < K; k += 32) mb = umax64(mb, abs_bits(at(k)));
    for (int o = 16; o > 0; o >>= 1) mb = umax64(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    const int e = row_exponent(__longlong_as_double((long long)mb));
    if (lane == 0) ex[warp] = e;
    const size_t plane = (size_t)R * K8;
    __nv_bfloat16* o = out + (size_t)warp * K8;
    for (int k = lane; k < K8; k += 32) {
        int d[MAX_S];
        if (k < K) digits(at(k), e, s, d);
        else
            for (int t = 0; t < MAX_S; ++t) d[t] = 0;
#pragma unroll
        for (int t = 0; t < MAX_S; ++t)
            if (t < s) o[t * plane + k] = slice_value(d[t], t);
    }
}

// General strides (rows contiguous when rs == 1).  Pass 1: per-row max|x|
// over K, the grid split over (32-row groups, K ranges), combined with
// atomicMax on the bit pattern.  Pass 2: a warp takes 32 rows x 32 k (lane =
// row while reading, so reads along contiguous rows coalesce), staged
// through shared memory so that the K-major slice writes coalesce too.
constexpr int COLS_KRANGE = 256;

__global__ void k_rowmax_cols(const double* __restrict__ X, int R, int K, View rv, View kv, int kranges,
                              unsigned long long* __restrict__ maxbits) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int rg = w / kranges, kr = w - rg * kranges;
    const int r = rg * 32 + lane;
    const int k0 = kr * COLS_KRANGE;
    if (r >= R || k0 >= K) return;
    const int k1 = min(K, k0 + COLS_KRANGE);
    const double* xr = X + view_offset32(rv, (unsigned)r);
    Odometer od;
    od.init(kv, (unsigned)k0);
    unsigned long long mx = 0;
    for (int k = k0; k < k1; k += 8) {
        long long off[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            off[u] = od.off;
            if (k + u + 1 < k1) od.step(kv);
        }
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (k + u < k1) ? xr[off[u]] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) mx = umax64(mx, abs_bits(v[u]));
    }
    atomicMax(maxbits + r, mx);
}

__global__ void k_split_cols(const double* __restrict__ X, int R, int K, int K8, View rv, View kv,
                             int s, const unsigned long long* __restrict__ maxbits, __nv_bfloat16* __restrict__ out,
                             int* __restrict__ ex) {
    __shared__ __nv_bfloat16 tile[2][MAX_S][32][33];  // launched with 2 warps
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * 32;
    const int k0 = (blockIdx.y * 2 + w) * 32;
    if (k0 >= K8) return;
    const int r = r0 + lane;
    const bool live = r < R;
    const int e = live ? row_exponent(__longlong_as_double((long long)maxbits[r])) : 0;
    if (live && k0 == 0) ex[r] = e;
    const double* xr = X + (live ? view_offset32(rv, (unsigned)r) : 0);
    Odometer od;
    od.init(kv, (unsigned)min(k0, K - 1));
    for (int kb = 0; kb < 32; kb += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + kb + u;
            v[u] = 0.0;
            if (live && k < K) {
                v[u] = xr[od.off];
                od.step(kv);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            int d[MAX_S];
            digits(v[u], e, s, d);
#pragma unroll
            for (int t = 0; t < MAX_S; ++t)
                if (t < s) tile[w][t][lane][kb + u] = slice_value(d[t], t);
        }
    }
    __syncwarp();
    const size_t plane = (size_t)R * K8;
    const int k = k0 + lane;
    if (k < K8)
        for (int rr = 0; rr < 32 && r0 + rr < R; ++rr)
            for (int t = 0; t < s; ++t) out[t * plane + (size_t)(r0 + rr) * K8 + k] = tile[w][t][rr][lane];
}

// round(x 2^(nbits - e)) as an integer, |x| <= 2^e (integer operations on the
// FP64 bit pattern, like digits())
__device__ __forceinline__ long long scaled_round(double x, int e, int nbits) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int ex = (int)((b >> 52) & 0x7ff);
    unsigned long long mant = b & ((1ull << 52) - 1);
    if (ex == 0) ex = 1;
    else mant |= 1ull << 52;
    const int shift = ex - 1075 + nbits - e;
    long long Y;
    if (mant == 0) Y = 0;
    else if (shift >= 0) Y = (long long)(mant << shift);
    else {
        const int sh = -shift;
        Y = sh >= 54 ? 0 : (long long)((mant + (1ull << (sh - 1))) >> sh);
    }
    return (b >> 63) ? -Y : Y;
}

// TF32 slices for 3xTF32: round(x 2^(22 - e)) = 2048 d0 + d1 with d1 in
// [-1024, 1023] and |d0| <= 2048; slice 0 = d0, slice 1 = d1 2^-11, each
// with at most 11 significant bits (exact in TF32), stored as FP32
// [2][R][K4].  One thread per row and 4 consecutive k (one 16-byte store per
// slice); general strided views; row maxima from k_rowmax_cols.
__global__ void k_split_tf32(const double* __restrict__ X, int R, int K, int K4, View rv, View kv,
                             const unsigned long long* __restrict__ maxbits, float* __restrict__ out,
                             int* __restrict__ ex) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nq = K4 / 4;
    const long long r = tid / nq;
    const int kq = (int)(tid - r * nq);
    if (r >= R) return;
    const int e = row_exponent(__longlong_as_double((long long)maxbits[r]));
    if (kq == 0) ex[r] = e;
    const long long roff = view_offset32(rv, (unsigned)r);
    float s0[4], s1[4];
    const float lo_scale = __int_as_float((127 - 11) << 23);  // 2^-11
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int k = 4 * kq + u;
        const double x = k < K ? X[roff + view_offset32(kv, (unsigned)k)] : 0.0;
        const int y = (int)scaled_round(x, e, 22);  // |y| <= 2^22
        const int hi = (y + 1024) >> 11;
        s0[u] = small_int_f32(hi);
        s1[u] = small_int_f32(y - (hi << 11)) * lo_scale;
    }
    const size_t plane = (size_t)R * K4;
    float* o = out + (size_t)r * K4 + 4 * kq;
    *reinterpret_cast<float4*>(o) = make_float4(s0[0], s0[1], s0[2], s0[3]);
    *reinterpret_cast<float4*>(o + plane) = make_float4(s1[0], s1[1], s1[2], s1[3]);
}

// ---------------------------------------------------------------------------
// Plain 2D operands (one row stride, one K stride): the slices of eight
// consecutive k of one row are built in registers and written as one 16-byte
// store per slice.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned bf2_bits(float a, float b) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);  // a in the low half (lower address)
    return *reinterpret_cast<const unsigned*>(&p);
}
// slice t of eight consecutive values as 8 BF16 (16 bytes), t < s
__device__ __forceinline__ void slice8_pack(const double* v, int e, int s, uint4* q) {
    int d[8][MAX_S];
#pragma unroll
    for (int u = 0; u < 8; ++u) digits(v[u], e, s, d[u]);
#pragma unroll
    for (int t = 0; t < MAX_S; ++t) {
        if (t < s) {
            const float sc = __int_as_float((127 - 8 * t) << 23);  // 2^(-8t)
            q[t].x = bf2_bits(small_int_f32(d[0][t]) * sc, small_int_f32(d[1][t]) * sc);
            q[t].y = bf2_bits(small_int_f32(d[2][t]) * sc, small_int_f32(d[3][t]) * sc);
            q[t].z = bf2_bits(small_int_f32(d[4][t]) * sc, small_int_f32(d[5][t]) * sc);
            q[t].w = bf2_bits(small_int_f32(d[6][t]) * sc, small_int_f32(d[7][t]) * sc);
        }
    }
}
// slice8_pack of eight FP64 bit patterns
__device__ __forceinline__ void slice8_pack_bits(const unsigned long long* vb, int e, int s, uint4* q) {
    int d[8][MAX_S];
#pragma unroll
    for (int u = 0; u < 8; ++u) digits_bits(vb[u], e, s, d[u]);
#pragma unroll
    for (int t = 0; t < MAX_S; ++t) {
        if (t < s) {
            const float sc = __int_as_float((127 - 8 * t) << 23);  // 2^(-8t)
            q[t].x = bf2_bits(small_int_f32(d[0][t]) * sc, small_int_f32(d[1][t]) * sc);
            q[t].y = bf2_bits(small_int_f32(d[2][t]) * sc, small_int_f32(d[3][t]) * sc);
            q[t].z = bf2_bits(small_int_f32(d[4][t]) * sc, small_int_f32(d[5][t]) * sc);
            q[t].w = bf2_bits(small_int_f32(d[6][t]) * sc, small_int_f32(d[7][t]) * sc);
        }
    }
}
__device__ __forceinline__ void slice8_store(const double* v, int e, int s, __nv_bfloat16* dst, size_t plane) {
    uint4 q[MAX_S];
    slice8_pack(v, e, s, q);
#pragma unroll
    for (int t = 0; t < MAX_S; ++t)
        if (t < s) *reinterpret_cast<uint4*>(dst + t * plane) = q[t];
}

// K contiguous, rows at stride rs, K8 <= 4 * 8 * TPR: TPR threads per row,
// each holding up to four 8-wide chunks (chunk c = j + i TPR) in registers,
// so X is read once.  VEC: rows start on 16 bytes (16-byte loads).
template <int TPR, bool VEC>
__global__ void __launch_bounds__(256) k_split_rows_reg(const double* __restrict__ X, int R, int K, int K8,
                                                       long long rs, int s, __nv_bfloat16* __restrict__ out,
                                                       int* __restrict__ ex) {
    constexpr int RPB = 256 / TPR;
    __shared__ unsigned long long red[8];
    const int g = threadIdx.x / TPR, j = threadIdx.x % TPR;
    const int r = blockIdx.x * RPB + g;
    const bool live = r < R;
    // the row is held as FP64 bit patterns: kept as doubles, every value
    // cost one FP64-pipe instruction (GB300 issues those at 2 lanes per
    // clock per SM), and nothing here needs FP64 arithmetic
    const unsigned long long* xr =
        reinterpret_cast<const unsigned long long*>(X) + (live ? (long long)r * rs : 0);
    const int nch = K8 >> 3;
    unsigned long long v[4][8];
    unsigned long long mb = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c = j + i * TPR;
        const int k0 = c * 8;
        if (VEC && live && c < nch && k0 + 8 <= K) {
            const ulonglong2* p2 = reinterpret_cast<const ulonglong2*>(xr + k0);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const ulonglong2 w = __ldcs(p2 + h);
                v[i][2 * h] = w.x;
                v[i][2 * h + 1] = w.y;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) v[i][u] = (live && c < nch && k0 + u < K) ? __ldcs(xr + k0 + u) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) mb = umax64(mb, v[i][u] & 0x7fffffffffffffffull);
    }
    if (TPR <= 32) {
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) mb = umax64(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mb = umax64(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) red[w] = mb;
        __syncthreads();
        constexpr int WPR = TPR / 32;  // warps per row
        mb = 0;
#pragma unroll
        for (int q = 0; q < WPR; ++q) mb = umax64(mb, red[g * WPR + q]);
    }
    if (!live) return;
    const int e = row_exponent_bits(mb);
    if (j == 0) ex[r] = e;
    const size_t plane = (size_t)R * K8;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c = j + i * TPR;
        if (c < nch) {
            uint4 q[MAX_S];
            slice8_pack_bits(v[i], e, s, q);
            __nv_bfloat16* dst = out + (size_t)r * K8 + (size_t)c * 8;
#pragma unroll
            for (int t = 0; t < MAX_S; ++t)
                if (t < s) *reinterpret_cast<uint4*>(dst + t * plane) = q[t];
        }
    }
}

// Rows contiguous (row stride 1), K at stride cs: lane = row, 32
// consecutive k per step (each load instruction reads 32 consecutive rows),
// one warp per 32 rows x kspan k (kspan a multiple of 32); row maxima from
// k_rowmax_cols.  The slices go out through shared memory so that four lanes
// write one row's 64 contiguous bytes in the same store instruction: lanes
// that each wrote 16 bytes of a different row left half-written sectors
// that L2 filled from DRAM (1.5x the bytes each way).
__global__ void __launch_bounds__(64) k_split_cols_reg(const double* __restrict__ X, int R, int K, int K8,
                                                      long long cs, int s,
                                                      const unsigned long long* __restrict__ maxbits,
                                                      __nv_bfloat16* __restrict__ out, int* __restrict__ ex,
                                                      int kspan, int kgroups) {
    // per warp: every slice of 32 rows x 4 x 16 bytes (+1 pad against bank conflicts)
    __shared__ uint4 tile[2][MAX_S][32][5];
    const int wid = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int rg = wid / kgroups, kg = wid - rg * kgroups;
    if (rg * 32 >= R) return;
    const int r0 = rg * 32, r = r0 + lane;
    const bool live = r < R;
    const int e = live ? row_exponent(__longlong_as_double((long long)maxbits[r])) : 0;
    if (live && kg == 0) ex[r] = e;
    const size_t plane = (size_t)R * K8;
    const int kend = min(K8, (kg + 1) * kspan);
    for (int k0 = kg * kspan; k0 < kend; k0 += 32) {
        double v[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) v[u] = (live && k0 + u < K) ? __ldcs(X + (long long)(k0 + u) * cs + r) : 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint4 q[MAX_S];
            slice8_pack(v + 8 * c, e, s, q);
#pragma unroll
            for (int t = 0; t < MAX_S; ++t)
                if (t < s) tile[w][t][lane][c] = q[t];
        }
        __syncwarp();
        // lane -> (row rr = j * 8 + lane / 4, 16-byte chunk c = lane % 4)
        for (int t = 0; t < s; ++t)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int rr = j * 8 + (lane >> 2), c = lane & 3;
                if (r0 + rr < R && k0 + 8 * c < kend)
                    *reinterpret_cast<uint4*>(out + t * plane + (size_t)(r0 + rr) * K8 + k0 + 8 * c) =
                        tile[w][t][rr][c];
            }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier, TMA, tcgen05
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or ~20 us pass, instead of spinning on issue slots
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `limit` cycles (about 1 s at the default
// 2e9), or at once when another thread has already given up, recording the
// failure in *err.
constexpr long long WAIT_LIMIT_CYCLES = 2000000000ll;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err,
                                          long long limit = WAIT_LIMIT_CYCLES) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*(volatile int*)err) return false;
        if (clock64() - t0 > limit) {
            atomicCAS(err, 0, 1);
            return false;
        }
    }
    return true;
}

// Failure-detection check of the bounded wait above: thread 0 waits on an
// mbarrier of count 1.  With `arrive` set, thread 32 arrives on it (the wait
// completes); without, nothing ever arrives and the wait must give up after
// `limit` cycles, set *err and return, leaving the context usable.
__global__ void k_wait_probe(long long limit, int arrive, int* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 32 && arrive) mbar_arrive(&bar);
    if (threadIdx.x == 0) mbar_wait(&bar, 0u, err, limit);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major, 64-byte-swizzled tile
// (rows of 64 bytes, 8-row groups 512 bytes apart).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;        // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)4 << 61;                 // SWIZZLE_64B
    return d;
}


// ---------------------------------------------------------------------------
// slice GEMM
// ---------------------------------------------------------------------------
struct GemmArgs {
    int M, N;             // logical output size
    int nkb;              // 32-wide k-blocks in K
    int kb_per_split;     // k-blocks per blockIdx.z (a multiple of CHUNK_KB)
    int s;                // slices per operand
    int stages;
    uint32_t a_bytes, stage_bytes;
    const int* eA;        // row exponents of A (M)
    const int* eB;        // column exponents of B (N)
    int direct;           // 1: write C; 0: write split-K partials
    double alpha, beta;
    double* C;
    View out_r, out_c;    // C offset of (m, n) = view(out_r, m) + view(out_c, n)
    int* PS0;             // split-K partials [z][Mpad][Npad]
    int* PS1;
    float* PF;
    int Mpad, Npad;
    int m_tiles, n_tiles;
    int* err;
    long long wait_limit; // cycles before a bounded wait gives up
};

// ONE: every CTA's K range is a single chunk (every corner product), so no
// sum is carried across chunks; a separate instantiation keeps the
// multi-chunk sums' registers out of that path.
// MODE 0: exact-level emulated FP64 (above).  MODE 1: split-BF16 -- the same
// BF16 digit slices, every product of levels <= s-1 accumulated in one FP32
// accumulator over all of K.  MODE 2: 3xTF32 -- two TF32 slices (base-2^11
// digits), hi*hi + hi*lo + lo*hi on kind::tf32 into one FP32 accumulator.
// Modes 1 and 2 run without split-K and read TMEM once per tile.
template <int NB16, bool ONE, int MODE>
__global__ void __launch_bounds__(THREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs g) {
    constexpr int BN = 16 * NB16;
    constexpr int NBG = (NB16 + 2) / 3;  // 16-column blocks per epilogue warp
    constexpr int NACC = MODE == 0 ? 3 : 1;  // TMEM accumulators of BN columns
    constexpr uint32_t TMEM_COLS = (NACC * BN <= 32) ? 32 : (NACC * BN <= 64) ? 64 : (NACC * BN <= 128) ? 128
                                   : (NACC * BN <= 256) ? 256 : 512;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sbase = smem_raw + (base - raw);
    uint64_t* full = (uint64_t*)(sbase + (size_t)g.stages * g.stage_bytes);
    uint64_t* empty = full + g.stages;
    uint64_t* acc_full = empty + g.stages;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* drain = acc_full + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Direct output: a persistent grid strides over the m_tiles x n_tiles
    // tiles, n fastest (CTAs running together share A tiles through L2), and
    // the stage ring and the accumulator hand-off run on across tiles, so one
    // tile's epilogue overlaps the next tile's loads and MMAs.  Split-K
    // partials: one tile per CTA (blockIdx x: m, y: n, z: split).
    const int ntiles = g.direct ? g.m_tiles * g.n_tiles : 1;
    const int t_first = g.direct ? (int)blockIdx.x : 0, t_step = g.direct ? (int)gridDim.x : 1;
    auto tile_m0 = [&](int t) { return (g.direct ? t / g.n_tiles : (int)blockIdx.x) * BM; };
    auto tile_n0 = [&](int t) { return (g.direct ? t % g.n_tiles : (int)blockIdx.y) * BN; };
    const int kb0 = g.direct ? 0 : (int)blockIdx.z * g.kb_per_split;
    const int kb1 = min(g.nkb, kb0 + g.kb_per_split);
    const int nkb = kb1 - kb0;
    const int nchunks = (nkb + CHUNK_KB - 1) / CHUNK_KB;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int st = 0; st < g.stages; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, EPI_WARPS);
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == EPI_WARPS) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int issued = 0;
            bool ok = true;
            for (int t = t_first; t < ntiles && ok; t += t_step) {
                const int m0 = tile_m0(t), n0 = tile_n0(t);
                for (int i = 0; i < nkb; ++i) {
                    const int st = issued % g.stages;
                    const uint32_t ph = (uint32_t)(issued / g.stages) & 1u;
                    if (!mbar_wait(&empty[st], ph ^ 1u, g.err, g.wait_limit)) {
                        ok = false;
                        break;
                    }
                    uint8_t* sa = sbase + (size_t)st * g.stage_bytes;
                    mbar_expect_tx(&full[st], g.stage_bytes);
                    const int kc = (kb0 + i) * (MODE == 2 ? BK / 2 : BK);  // 64 bytes of K per stage
                    tma_load_3d(sa, &tmA, kc, m0, 0, &full[st]);
                    tma_load_3d(sa + g.a_bytes, &tmB, kc, n0, 0, &full[st]);
                    ++issued;
                }
            }
            if (*(volatile int*)g.err) {
                // let the copies still in flight land before the CTA exits
                for (int i = max(0, issued - g.stages); i < issued; ++i) {
                    const long long t0 = clock64();
                    while (!mbar_try_wait(&full[i % g.stages], (uint32_t)(i / g.stages) & 1u) &&
                           clock64() - t0 < g.wait_limit) {
                    }
                }
            }
        }
    } else if (warp == EPI_WARPS + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            // D format F32 (1); A and B both BF16 (1) under kind::f16, both TF32 (2) under kind::tf32
            constexpr uint32_t fmt = MODE == 2 ? 2u : 1u;
            const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) |
                                   ((uint32_t)(BM >> 4) << 24);
            int it = 0, cc = 0;  // k-blocks and accumulator chunks issued so far, over all tiles
            bool ok = true;
            for (int t = t_first; t < ntiles && ok; t += t_step)
            for (int i = 0; i < nkb; ++i, ++it) {
                const int st = it % g.stages;
                const uint32_t ph = (uint32_t)(it / g.stages) & 1u;
                const bool first = MODE == 0 ? (i % CHUNK_KB) == 0 : i == 0;
                const bool last = MODE == 0 ? ((i % CHUNK_KB) == CHUNK_KB - 1 || i == nkb - 1) : i == nkb - 1;
                if (first && cc > 0 && !mbar_wait(acc_empty, (uint32_t)(cc - 1) & 1u, g.err, g.wait_limit)) {
                    ok = false;
                    break;
                }
                if (!mbar_wait(&full[st], ph, g.err, g.wait_limit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = base + (uint32_t)st * g.stage_bytes;
                const uint32_t sb = sa + g.a_bytes;
                if (MODE != 0) {
                    // two 32-byte K halves (16 BF16 or 8 TF32 each); every level
                    // <= s-1 into the one FP32 accumulator
                    for (int h = 0; h < 2; ++h) {
                        bool f1 = first && h == 0;
                        for (int L = 0; L < g.s; ++L)
                            for (int t = 0; t <= L; ++t) {
                                const uint64_t ad = sw64_desc(sa + t * (BM * 64) + h * 32);
                                const uint64_t bd = sw64_desc(sb + (L - t) * (BN * 64) + h * 32);
                                if (MODE == 2) tc_mma_tf32(tmem, ad, bd, idesc, f1 ? 0u : 1u);
                                else tc_mma(tmem, ad, bd, idesc, f1 ? 0u : 1u);
                                f1 = false;
                            }
                    }
                } else
                for (int h = 0; h < 2; ++h) {  // two K=16 halves, 32 bytes apart in the 64-byte row
                    const uint32_t restart = (first && h == 0) ? 0u : 1u;
                    tc_mma(tmem, sw64_desc(sa + h * 32), sw64_desc(sb + h * 32), idesc, restart);
                    tc_mma(tmem + BN, sw64_desc(sa + h * 32), sw64_desc(sb + BN * 64 + h * 32), idesc, restart);
                    tc_mma(tmem + BN, sw64_desc(sa + BM * 64 + h * 32), sw64_desc(sb + h * 32), idesc, 1u);
                    bool first2 = first && h == 0;  // the FP32 levels restart every chunk
                    for (int L = 2; L < g.s; ++L)
                        for (int t = 0; t <= L; ++t) {
                            tc_mma(tmem + 2 * BN, sw64_desc(sa + t * (BM * 64) + h * 32),
                                   sw64_desc(sb + (L - t) * (BN * 64) + h * 32), idesc, first2 ? 0u : 1u);
                            first2 = false;
                        }
                }
                tc_commit(&empty[st]);
                if (last) {
                    tc_commit(acc_full);
                    ++cc;
                }
            }
            // every MMA issued by this thread completes before TMEM is freed
            tc_commit(drain);
            const long long t0 = clock64();
            while (!mbar_try_wait(drain, 0u) && clock64() - t0 < g.wait_limit) {
            }
        }
    } else if (MODE != 0) {
        // ---------------- epilogue of the FP32-accumulated modes ----------------
        const int q = warp & 3, grp = warp >> 2;
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
        const bool unit_alpha = g.alpha == 1.0, zero_beta = g.beta == 0.0;
        constexpr int dbits = MODE == 2 ? 11 : 8;  // digit width of the slices
        int cc = 0;
        for (int t = t_first; t < ntiles; t += t_step, ++cc) {
            const int m0 = tile_m0(t), n0 = tile_n0(t);
            const int m = m0 + q * 32 + lane;
            const int ea = m < g.M ? g.eA[m] : 0;
            if (!mbar_wait(acc_full, (uint32_t)cc & 1u, g.err, g.wait_limit)) break;
            tc_fence_after();
            float F[NBG][16];
#pragma unroll
            for (int jb = 0; jb < NBG; ++jb) {
                const int b = grp + 3 * jb;
                if (b >= NB16) continue;
                uint32_t r[16];
                tc_ld16(lane_addr + b * 16, r);
                tc_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) F[jb][j] = __uint_as_float(r[j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty);
#pragma unroll
            for (int jb = 0; jb < NBG; ++jb) {
                const int b = grp + 3 * jb;
                if (b >= NB16) continue;
                const int nl = n0 + b * 16 + (lane & 15);
                const long long coff_l = nl < g.N ? view_offset32(g.out_c, (unsigned)nl) : 0;
                const int eb_l = nl < g.N ? g.eB[nl] : 0;
                double* crow = g.C + (m < g.M ? view_offset32(g.out_r, (unsigned)m) : 0);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const long long coff = __shfl_sync(0xffffffffu, coff_l, j);
                    const int eb = __shfl_sync(0xffffffffu, eb_l, j);
                    const int n = n0 + b * 16 + j;
                    if (m >= g.M || n >= g.N) continue;
                    double v = f32_scaled(F[jb][j], ea + eb - 2 * dbits);
                    if (ea > 1024 || eb > 1024) v = __longlong_as_double(0x7ff8000000000000ll);  // non-finite operand
                    double* cp = crow + coff;
                    // uniform branch: no FP64 arithmetic issued when alpha = 1, beta = 0
                    if (unit_alpha && zero_beta) *cp = v;
                    else *cp = zero_beta ? v * g.alpha : fma(g.beta, *cp, v * g.alpha);
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 0..11 ----------------
        const int q = warp & 3, grp = warp >> 2;
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
        int cc = 0;  // accumulator chunks drained so far, over all tiles
        bool ok = true;
        const bool unit_alpha = g.alpha == 1.0, zero_beta = g.beta == 0.0;
        for (int t = t_first; t < ntiles && ok; t += t_step) {
        const int m0 = tile_m0(t), n0 = tile_n0(t);
        const int m = m0 + q * 32 + lane;
        const int ea = (g.direct && m < g.M) ? g.eA[m] : 0;
        // Multi-chunk tiles carry the exact level-0/1 sums (int32) and the
        // sum of the per-chunk FP32 levels across K chunks, and finish each
        // 16-column block in the last chunk before reading the next.  A
        // single-chunk tile (every corner product: K <= 256) reads all of
        // TMEM first and releases it, so that the next tile's MMAs run while
        // this tile's results are assembled and stored.
        constexpr int NC = NBG;
        int S0[NC][16], S1[NC][16];
        float Fs[NC][16];
#pragma unroll
        for (int jb = 0; jb < NC; ++jb)
#pragma unroll
            for (int j = 0; j < 16; ++j) S0[jb][j] = S1[jb][j] = 0, Fs[jb][j] = 0.f;
        // result of column block jb: assembled and stored (direct) or kept
        // as split-K partials
        auto finish = [&](int jb) {
            const int b = grp + 3 * jb;
            if (g.direct) {
                // the 16 columns of this block are the same for every lane:
                // lane j works out column j's offset and exponent once
                const int nl = n0 + b * 16 + (lane & 15);
                const long long coff_l = nl < g.N ? view_offset32(g.out_c, (unsigned)nl) : 0;
                const int eb_l = nl < g.N ? g.eB[nl] : 0;
                double* crow = g.C + (m < g.M ? view_offset32(g.out_r, (unsigned)m) : 0);
                // alpha = 1, beta = 0 (every product of the sweep) takes a loop
                // with no FP64 arithmetic at all: the branch is uniform, so
                // the scaling is not issued under a predicate per element
                if (unit_alpha && zero_beta) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const long long coff = __shfl_sync(0xffffffffu, coff_l, j);
                        const int eb = __shfl_sync(0xffffffffu, eb_l, j);
                        const int n = n0 + b * 16 + j;
                        if (m >= g.M || n >= g.N) continue;
                        double v = assemble(S0[jb][j], S1[jb][j], Fs[jb][j], ea + eb - 16);
                        if (ea > 1024 || eb > 1024) v = __longlong_as_double(0x7ff8000000000000ll);  // non-finite operand
                        crow[coff] = v;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const long long coff = __shfl_sync(0xffffffffu, coff_l, j);
                        const int eb = __shfl_sync(0xffffffffu, eb_l, j);
                        const int n = n0 + b * 16 + j;
                        if (m >= g.M || n >= g.N) continue;
                        double v = assemble(S0[jb][j], S1[jb][j], Fs[jb][j], ea + eb - 16);
                        if (ea > 1024 || eb > 1024) v = __longlong_as_double(0x7ff8000000000000ll);
                        v *= g.alpha;
                        double* cp = crow + coff;
                        *cp = zero_beta ? v : fma(g.beta, *cp, v);
                    }
                }
            } else {
                const size_t row = ((size_t)blockIdx.z * g.Mpad + m) * g.Npad + n0 + b * 16;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    g.PS0[row + j] = S0[jb][j];
                    g.PS1[row + j] = S1[jb][j];
                    g.PF[row + j] = Fs[jb][j];
                }
            }
        };
        for (int c = 0; c < nchunks; ++c, ++cc) {
            if (!mbar_wait(acc_full, (uint32_t)cc & 1u, g.err, g.wait_limit)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const bool last = c == nchunks - 1;
#pragma unroll
            for (int jb = 0; jb < NBG; ++jb) {
                const int b = grp + 3 * jb;
                if (b >= NB16) continue;
                uint32_t r0[16], r1[16];
                tc_ld16(lane_addr + b * 16, r0);
                tc_ld16(lane_addr + BN + b * 16, r1);
                tc_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    S0[jb][j] += __float2int_rn(__uint_as_float(r0[j]));
                    S1[jb][j] += __float2int_rn(__uint_as_float(r1[j]) * 256.0f);
                }
                if (g.s > 2) {
                    tc_ld16(lane_addr + 2 * BN + b * 16, r0);
                    tc_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) Fs[jb][j] += __uint_as_float(r0[j]);
                }
                if (!ONE && last) finish(jb);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty);
        }
        if (ONE && ok) {
#pragma unroll
            for (int jb = 0; jb < NBG; ++jb)
                if (grp + 3 * jb < NB16) finish(jb);
        }
        }  // tiles
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// split-K partials -> C
__global__ void k_oz_combine(const int* __restrict__ PS0, const int* __restrict__ PS1, const float* __restrict__ PF,
                             int splits, int Mpad, int Npad, int M, int N, const int* __restrict__ eA,
                             const int* __restrict__ eB, double alpha, double beta, double* __restrict__ C,
                             View out_r, View out_c) {
    const size_t total = (size_t)M * N;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(t / N), n = (int)(t % N);
        // split-K runs only for small outputs: FP64 sums here are cheap and
        // cannot overflow however many splits there are
        double v = 0.0;
        for (int z = 0; z < splits; ++z) {
            const size_t idx = ((size_t)z * Mpad + m) * Npad + n;
            const long long T = (long long)PS0[idx] * 256 + (long long)PS1[idx];
            v += (double)T + (double)(PF[idx] * 256.0f);
        }
        v = (eA[m] > 1024 || eB[n] > 1024) ? __longlong_as_double(0x7ff8000000000000ll)  // non-finite operand
                                           : scale_pow2(v, eA[m] + eB[n] - 24);
        if (alpha != 1.0) v *= alpha;
        double* cp = C + view_offset32(out_r, (unsigned)m) + view_offset32(out_c, (unsigned)n);
        *cp = (beta == 0.0) ? v : fma(beta, *cp, v);
    }
}

}  // namespace oz
}  // namespace ctm

// ===========================================================================
// host side
// ===========================================================================
namespace ctm {
namespace {

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
inline int k8_of(int K) { return (K + 7) & ~7; }
inline int k4_of(int K) { return (K + 3) & ~3; }

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// slices [s][R][Kp], 64-byte-swizzled boxes of {64 bytes of k, rows, s}:
// BF16 (Kp = K8, 32 k per box row) or TF32 as FP32 (Kp = K4, 16 k)
bool make_map(CUtensorMap* map, const void* slices, int R, int Kp, int s, int box_rows, bool tf32 = false) {
    auto enc = tmap_encoder();
    if (!enc) return false;
    const int esz = tf32 ? 4 : 2;
    const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)R, (cuuint64_t)s};
    const cuuint64_t strides[2] = {(cuuint64_t)Kp * esz, (cuuint64_t)R * Kp * esz};
    const cuuint32_t box[3] = {(cuuint32_t)(64 / esz), (cuuint32_t)box_rows, (cuuint32_t)s};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
               const_cast<void*>(slices), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Plan {
    int nb16, bn, m_tiles, n_tiles, ksplit, kb_per_split, nkb, stages;
    uint32_t a_bytes, stage_bytes;
    size_t smem, ws_bytes;
};

// mode 2 (3xTF32) holds 16 k per 64-byte stage row instead of 32; modes 1 and
// 2 never split K
Plan plan_of(int M, int N, int K, int s, int mode = 0) {
    Plan p{};
    // fewest 144-wide tiles, then the narrowest 16-multiple width that covers N
    const int nt = (N + 143) / 144;
    p.nb16 = ((N + nt - 1) / nt + 15) / 16;
    if (p.nb16 < 1) p.nb16 = 1;
    p.bn = 16 * p.nb16;
    p.m_tiles = (M + oz::BM - 1) / oz::BM;
    p.n_tiles = (N + p.bn - 1) / p.bn;
    p.nkb = mode == 2 ? (k4_of(K) + 15) / 16 : (k8_of(K) + oz::BK - 1) / oz::BK;
    if (p.nkb < 1) p.nkb = 1;
    const int nchunks = (p.nkb + oz::CHUNK_KB - 1) / oz::CHUNK_KB;
    const int tiles = p.m_tiles * p.n_tiles;
    int ks = 1;
    if (mode == 0 && tiles < 120 && nchunks >= 2) ks = std::min(nchunks, (148 + tiles - 1) / tiles);
    // int32 level sums stay exact for K <= 16384 per split
    const int max_chunks_per_split = 16384 / (oz::CHUNK_KB * oz::BK);
    if (mode == 0) ks = std::max(ks, (nchunks + max_chunks_per_split - 1) / max_chunks_per_split);
    const int cps = (nchunks + ks - 1) / ks;
    p.kb_per_split = mode == 0 ? cps * oz::CHUNK_KB : p.nkb;
    p.ksplit = (p.nkb + p.kb_per_split - 1) / p.kb_per_split;
    p.a_bytes = (uint32_t)(s * oz::BM * oz::BK * 2);
    p.stage_bytes = p.a_bytes + (uint32_t)(s * p.bn * oz::BK * 2);
    p.stages = std::min<int>(6, (int)((220u * 1024u) / p.stage_bytes));
    p.smem = (size_t)p.stages * p.stage_bytes + 1024 + 256;
    p.ws_bytes = p.ksplit > 1 ? 3 * align256((size_t)p.ksplit * p.m_tiles * oz::BM * p.n_tiles * p.bn * 4) : 0;
    return p;
}

template <int NB16, bool ONE, int MODE = 0>
cudaError_t launch_gemm(const Plan& p, const CUtensorMap& ta, const CUtensorMap& tb, const oz::GemmArgs& g,
                        cudaStream_t st) {
    // the 227 KB dynamic shared-memory opt-in is a per-device function
    // attribute: set it once for every device this instantiation runs on
    static std::mutex mu;
    static unsigned long long done = 0;  // bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!(done >> dev & 1ull)) {
            e = cudaFuncSetAttribute(oz::k_oz_gemm<NB16, ONE, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     227 * 1024);
            if (e != cudaSuccess) return e;
            done |= 1ull << dev;
        }
    }
    dim3 grid(p.m_tiles, p.n_tiles, p.ksplit);
    if (g.direct) {
        // persistent: one CTA per SM (the stage ring fills shared memory)
        int nsm = 0;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const long long tiles = (long long)p.m_tiles * p.n_tiles;
        grid = dim3((unsigned)std::min<long long>(tiles, nsm > 0 ? nsm : 1), 1, 1);
    }
    ++g_launches;
    oz::k_oz_gemm<NB16, ONE, MODE><<<grid, oz::THREADS, p.smem, st>>>(ta, tb, g);
    return cudaGetLastError();
}

}  // namespace

// split buffer: slices [s][R][K8] | row max bits [R] (u64) | exponents [R] (int)
size_t oz_split_bytes(int R, int K, int s) {
    return align256((size_t)s * R * k8_of(K) * 2) + align256((size_t)R * 8) + align256((size_t)R * 4);
}
inline const int* split_exponents(const void* buf, int R, int K8, int s) {
    return (const int*)((const char*)buf + align256((size_t)s * R * K8 * 2) + align256((size_t)R * 8));
}
// TF32 split buffer: slices [2][R][K4] (FP32) | row max bits [R] | exponents [R]
size_t oz_split_tf32_bytes(int R, int K) {
    return align256((size_t)2 * R * k4_of(K) * 4) + align256((size_t)R * 8) + align256((size_t)R * 4);
}
inline const int* split_tf32_exponents(const void* buf, int R, int K4) {
    return (const int*)((const char*)buf + align256((size_t)2 * R * K4 * 4) + align256((size_t)R * 8));
}

cudaError_t oz_split_tf32(const double* X, int R, int K, const OzView& rvh, const OzView& kvh, void* buf,
                          cudaStream_t st) {
    if (R <= 0 || K <= 0 || rvh.n < 1 || rvh.n > 4 || kvh.n < 1 || kvh.n > 4) return cudaErrorInvalidValue;
    oz::View rv, kv;
    rv.n = rvh.n;
    kv.n = kvh.n;
    for (int a = 0; a < 4; ++a) {
        rv.dim[a] = rvh.dim[a];
        rv.stride[a] = rvh.stride[a];
        kv.dim[a] = kvh.dim[a];
        kv.stride[a] = kvh.stride[a];
    }
    const int K4 = k4_of(K);
    float* sl = (float*)buf;
    unsigned long long* mb = (unsigned long long*)((char*)buf + align256((size_t)2 * R * K4 * 4));
    int* ex = const_cast<int*>(split_tf32_exponents(buf, R, K4));
    cudaError_t e = cudaMemsetAsync(mb, 0, (size_t)R * 8, st);
    if (e != cudaSuccess) return e;
    const unsigned rg = (unsigned)((R + 31) / 32);
    const unsigned kr = (unsigned)((K + oz::COLS_KRANGE - 1) / oz::COLS_KRANGE);
    const unsigned long long warps = (unsigned long long)rg * kr;
    const unsigned long long threads = (unsigned long long)R * (K4 / 4);
    if ((warps + 3) / 4 > 0x7fffffffull || (threads + 255) / 256 > 0x7fffffffull) return cudaErrorInvalidValue;
    ++g_launches;
    oz::k_rowmax_cols<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(X, R, K, rv, kv, (int)kr, mb);
    ++g_launches;
    oz::k_split_tf32<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(X, R, K, K4, rv, kv, mb, sl, ex);
    return cudaGetLastError();
}

template <int TPR>
void launch_rows_reg_t(bool vec, unsigned blocks, cudaStream_t st, const double* X, int R, int K, int K8,
                       long long rs, int s, __nv_bfloat16* sl, int* ex) {
    if (vec) oz::k_split_rows_reg<TPR, true><<<blocks, 256, 0, st>>>(X, R, K, K8, rs, s, sl, ex);
    else oz::k_split_rows_reg<TPR, false><<<blocks, 256, 0, st>>>(X, R, K, K8, rs, s, sl, ex);
}
void launch_split_rows_reg(int tpr, bool vec, unsigned blocks, cudaStream_t st, const double* X, int R, int K,
                           int K8, long long rs, int s, __nv_bfloat16* sl, int* ex) {
    switch (tpr) {
        case 1: launch_rows_reg_t<1>(vec, blocks, st, X, R, K, K8, rs, s, sl, ex); break;
        case 2: launch_rows_reg_t<2>(vec, blocks, st, X, R, K, K8, rs, s, sl, ex); break;
        case 4: launch_rows_reg_t<4>(vec, blocks, st, X, R, K, K8, rs, s, sl, ex); break;
        case 8: launch_rows_reg_t<8>(vec, blocks, st, X, R, K, K8, rs, s, sl, ex); break;
        case 16: launch_rows_reg_t<16>(vec, blocks, st, X, R, K, K8, rs, s, sl, ex); break;
        case 32: launch_rows_reg_t<32>(vec, blocks, st, X, R, K, K8, rs, s, sl, ex); break;
        case 64: launch_rows_reg_t<64>(vec, blocks, st, X, R, K, K8, rs, s, sl, ex); break;
        case 128: launch_rows_reg_t<128>(vec, blocks, st, X, R, K, K8, rs, s, sl, ex); break;
        default: launch_rows_reg_t<256>(vec, blocks, st, X, R, K, K8, rs, s, sl, ex); break;
    }
}

cudaError_t oz_split(const double* X, int R, int K, long long rs, long long cs, int s, void* buf, cudaStream_t st) {
    OzView rv{1, {R, 1, 1, 1}, {rs, 0, 0, 0}}, kv{1, {K, 1, 1, 1}, {cs, 0, 0, 0}};
    return oz_split_view(X, R, K, rv, kv, s, buf, st);
}

cudaError_t oz_split_view(const double* X, int R, int K, const OzView& rvh, const OzView& kvh, int s, void* buf,
                          cudaStream_t st) {
    if (R <= 0 || K <= 0 || s < 2 || s > oz::MAX_S || rvh.n < 1 || rvh.n > 4 || kvh.n < 1 || kvh.n > 4)
        return cudaErrorInvalidValue;
    oz::View rv, kv;
    rv.n = rvh.n;
    kv.n = kvh.n;
    for (int a = 0; a < 4; ++a) {
        rv.dim[a] = rvh.dim[a];
        rv.stride[a] = rvh.stride[a];
        kv.dim[a] = kvh.dim[a];
        kv.stride[a] = kvh.stride[a];
    }
    const long long cs = kv.stride[kv.n - 1];
    const int K8 = k8_of(K);
    __nv_bfloat16* sl = (__nv_bfloat16*)buf;
    unsigned long long* mb = (unsigned long long*)((char*)buf + align256((size_t)s * R * K8 * 2));
    int* ex = const_cast<int*>(split_exponents(buf, R, K8, s));
    const int nch = K8 / 8;
    if (cs == 1 && rv.n == 1 && kv.n == 1 && nch <= 4 * 256) {
        int tpr = 1;
        while (tpr * 4 < nch) tpr *= 2;
        const bool vec = ((uintptr_t)X % 16 == 0) && (rv.stride[0] % 2 == 0);
        const unsigned blocks = (unsigned)(((size_t)R * tpr + 255) / 256);
        ++g_launches;
        launch_split_rows_reg(tpr, vec, blocks, st, X, R, K, K8, rv.stride[0], s, sl, ex);
    } else if (cs == 1) {
        ++g_launches;
        const unsigned blocks = (unsigned)(((size_t)R * 32 + 255) / 256);
        oz::k_split_rows<<<blocks, 256, 0, st>>>(X, R, K, K8, rv, kv, s, sl, ex);
    } else if (rv.n == 1 && rv.stride[0] == 1 && kv.n == 1) {
        cudaError_t e = cudaMemsetAsync(mb, 0, (size_t)R * 8, st);
        if (e != cudaSuccess) return e;
        const unsigned rg = (unsigned)((R + 31) / 32);
        const unsigned kr = (unsigned)((K + oz::COLS_KRANGE - 1) / oz::COLS_KRANGE);
        const unsigned long long warps = (unsigned long long)rg * kr;
        const int kspan = 256, kgroups = (K8 + kspan - 1) / kspan;
        const unsigned long long warps2 = (unsigned long long)rg * kgroups;
        if ((warps + 3) / 4 > 0x7fffffffull || (warps2 + 1) / 2 > 0x7fffffffull) return cudaErrorInvalidValue;
        ++g_launches;
        oz::k_rowmax_cols<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(X, R, K, rv, kv, (int)kr, mb);
        ++g_launches;
        oz::k_split_cols_reg<<<(unsigned)((warps2 + 1) / 2), 64, 0, st>>>(X, R, K, K8, kv.stride[0], s, mb, sl, ex,
                                                                           kspan, kgroups);
    } else {
        cudaError_t e = cudaMemsetAsync(mb, 0, (size_t)R * 8, st);
        if (e != cudaSuccess) return e;
        const unsigned rg = (unsigned)((R + 31) / 32);
        const unsigned kr = (unsigned)((K + oz::COLS_KRANGE - 1) / oz::COLS_KRANGE);
        const unsigned long long warps = (unsigned long long)rg * kr;
        if ((warps + 3) / 4 > 0x7fffffffull || (K8 / 32 + 2) / 2 > 65535) return cudaErrorInvalidValue;
        ++g_launches;
        oz::k_rowmax_cols<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(X, R, K, rv, kv, (int)kr, mb);
        ++g_launches;
        oz::k_split_cols<<<dim3(rg, (unsigned)((K8 / 32 + 1 + 1) / 2)), 64, 0, st>>>(X, R, K, K8, rv, kv, s, mb, sl, ex);
    }
    return cudaGetLastError();
}

cudaError_t wait_probe(long long limit_cycles, int arrive, int* err, cudaStream_t st) {
    ++g_launches;
    oz::k_wait_probe<<<1, 64, 0, st>>>(limit_cycles, arrive, err);
    return cudaGetLastError();
}

size_t oz_gemm_ws_bytes(int M, int N, int K, int s, int mode) { return plan_of(M, N, K, s, mode).ws_bytes; }

cudaError_t oz_gemm(int M, int N, int K, int s, const void* Asplit, const void* Bsplit, double alpha, double beta,
                    double* C, int ldc, void* ws, size_t ws_bytes, int* err, cudaStream_t st, int mode) {
    OzView r{1, {M, 1, 1, 1}, {ldc, 0, 0, 0}}, c{1, {N, 1, 1, 1}, {1, 0, 0, 0}};
    return oz_gemm_view(M, N, K, s, Asplit, Bsplit, alpha, beta, C, r, c, ws, ws_bytes, err, st, mode);
}

cudaError_t oz_gemm_view(int M, int N, int K, int s, const void* Asplit, const void* Bsplit, double alpha,
                         double beta, double* C, const OzView& orv, const OzView& ocv, void* ws, size_t ws_bytes,
                         int* err, cudaStream_t st, int mode) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K <= 0 || s < 2 || s > oz::MAX_S || mode < 0 || mode > 2 || (mode == 2 && s != 2))
        return cudaErrorInvalidValue;
    const Plan p = plan_of(M, N, K, s, mode);
    if (p.stages < 2 || p.ws_bytes > ws_bytes) return cudaErrorInvalidValue;
    const int Kp = mode == 2 ? k4_of(K) : k8_of(K);
    CUtensorMap ta, tb;
    if (!make_map(&ta, Asplit, M, Kp, s, oz::BM, mode == 2) || !make_map(&tb, Bsplit, N, Kp, s, p.bn, mode == 2))
        return cudaErrorInvalidValue;
    oz::GemmArgs g{};
    g.M = M;
    g.N = N;
    g.nkb = p.nkb;
    g.kb_per_split = p.kb_per_split;
    g.s = s;
    g.stages = p.stages;
    g.a_bytes = p.a_bytes;
    g.stage_bytes = p.stage_bytes;
    g.eA = mode == 2 ? split_tf32_exponents(Asplit, M, Kp) : split_exponents(Asplit, M, Kp, s);
    g.eB = mode == 2 ? split_tf32_exponents(Bsplit, N, Kp) : split_exponents(Bsplit, N, Kp, s);
    g.direct = p.ksplit == 1;
    g.alpha = alpha;
    g.beta = beta;
    g.C = C;
    g.out_r.n = orv.n;
    g.out_c.n = ocv.n;
    for (int a = 0; a < 4; ++a) {
        g.out_r.dim[a] = orv.dim[a];
        g.out_r.stride[a] = orv.stride[a];
        g.out_c.dim[a] = ocv.dim[a];
        g.out_c.stride[a] = ocv.stride[a];
    }
    g.Mpad = p.m_tiles * oz::BM;
    g.m_tiles = p.m_tiles;
    g.n_tiles = p.n_tiles;
    g.Npad = p.n_tiles * p.bn;
    if (!g.direct) {
        const size_t part = align256((size_t)p.ksplit * g.Mpad * g.Npad * 4);
        g.PS0 = (int*)ws;
        g.PS1 = (int*)((char*)ws + part);
        g.PF = (float*)((char*)ws + 2 * part);
    }
    g.err = err;
    g.wait_limit = oz::WAIT_LIMIT_CYCLES;
    // a CTA's K range: all of K (direct) or kb_per_split k-blocks (split-K)
    const bool one = (p.ksplit == 1 ? p.nkb : p.kb_per_split) <= oz::CHUNK_KB;
    cudaError_t e;
    if (mode != 0) {
        switch (p.nb16 * 4 + mode) {
            case 5: e = launch_gemm<1, true, 1>(p, ta, tb, g, st); break;
            case 6: e = launch_gemm<1, true, 2>(p, ta, tb, g, st); break;
            case 9: e = launch_gemm<2, true, 1>(p, ta, tb, g, st); break;
            case 10: e = launch_gemm<2, true, 2>(p, ta, tb, g, st); break;
            case 13: e = launch_gemm<3, true, 1>(p, ta, tb, g, st); break;
            case 14: e = launch_gemm<3, true, 2>(p, ta, tb, g, st); break;
            case 17: e = launch_gemm<4, true, 1>(p, ta, tb, g, st); break;
            case 18: e = launch_gemm<4, true, 2>(p, ta, tb, g, st); break;
            case 21: e = launch_gemm<5, true, 1>(p, ta, tb, g, st); break;
            case 22: e = launch_gemm<5, true, 2>(p, ta, tb, g, st); break;
            case 25: e = launch_gemm<6, true, 1>(p, ta, tb, g, st); break;
            case 26: e = launch_gemm<6, true, 2>(p, ta, tb, g, st); break;
            case 29: e = launch_gemm<7, true, 1>(p, ta, tb, g, st); break;
            case 30: e = launch_gemm<7, true, 2>(p, ta, tb, g, st); break;
            case 33: e = launch_gemm<8, true, 1>(p, ta, tb, g, st); break;
            case 34: e = launch_gemm<8, true, 2>(p, ta, tb, g, st); break;
            case 37: e = launch_gemm<9, true, 1>(p, ta, tb, g, st); break;
            default: e = launch_gemm<9, true, 2>(p, ta, tb, g, st); break;
        }
        return e;
    }
    switch (p.nb16 * 2 + (one ? 1 : 0)) {
        case 2: e = launch_gemm<1, false>(p, ta, tb, g, st); break;
        case 3: e = launch_gemm<1, true>(p, ta, tb, g, st); break;
        case 4: e = launch_gemm<2, false>(p, ta, tb, g, st); break;
        case 5: e = launch_gemm<2, true>(p, ta, tb, g, st); break;
        case 6: e = launch_gemm<3, false>(p, ta, tb, g, st); break;
        case 7: e = launch_gemm<3, true>(p, ta, tb, g, st); break;
        case 8: e = launch_gemm<4, false>(p, ta, tb, g, st); break;
        case 9: e = launch_gemm<4, true>(p, ta, tb, g, st); break;
        case 10: e = launch_gemm<5, false>(p, ta, tb, g, st); break;
        case 11: e = launch_gemm<5, true>(p, ta, tb, g, st); break;
        case 12: e = launch_gemm<6, false>(p, ta, tb, g, st); break;
        case 13: e = launch_gemm<6, true>(p, ta, tb, g, st); break;
        case 14: e = launch_gemm<7, false>(p, ta, tb, g, st); break;
        case 15: e = launch_gemm<7, true>(p, ta, tb, g, st); break;
        case 16: e = launch_gemm<8, false>(p, ta, tb, g, st); break;
        case 17: e = launch_gemm<8, true>(p, ta, tb, g, st); break;
        case 18: e = launch_gemm<9, false>(p, ta, tb, g, st); break;
        default: e = launch_gemm<9, true>(p, ta, tb, g, st); break;
    }
    if (e != cudaSuccess || g.direct) return e;
    size_t blocks = ((size_t)M * N + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    ++g_launches;
    oz::k_oz_combine<<<(unsigned)blocks, 256, 0, st>>>(g.PS0, g.PS1, g.PF, p.ksplit, g.Mpad, g.Npad, M, N, g.eA,
                                                        g.eB, alpha, beta, C, g.out_r, g.out_c);
    return cudaGetLastError();
}

}  // namespace ctm
