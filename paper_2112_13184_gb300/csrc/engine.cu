// CTMRG engine and C ABI (include/ctm.h).
//
// The sweep (Sec. 2.2) is built from one routine: the enlarged corner
//   E(C, T, T', A)[(a,d,d'), (b,r,r')] = sum C[g,h] T[h,u,u',b] T'[a,l,l',g]
//                                        A[s,l,u,r,d] A[s,l',u',r',d'],
// the upper-left corner of a site.  The other three corners are the same
// routine on the lattice rotated by 90, 180, 270 degrees counter-clockwise:
// corner c of a site is E(C_c, T_c, T_{c-1}, rot^c A), rot(A)[s,l,u,r,d] =
// A[s,d,l,u,r], with the corners/edges numbered clockwise (C1 T1 C2 T2 ...).
// A left move on the frame rotated m times is the move in direction m.
//
// Projectors of a cut (QR-free, Sec. 2.2): with H_u = Q_ul Q_ur, H_d = Q_bl Q_br
// and M = H_u^T H_d, the top-chi SVD M ~ U S V^T is taken by a randomised
// range finder (Halko et al.) that only applies M and M^T as chains of four
// corner products -- M is never formed:
//   M X   = E_ur^T E_ul^T E_bl^T E_br^T X,   M^T X = E_br E_bl E_ul E_ur X,
//   P_up  = E_bl^T E_br^T V S^{-1/2},        P_dn^T = E_ul E_ur U S^{-1/2}.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <set>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace ctm;

namespace {

enum { C1 = 0, T1 = 1, C2 = 2, T2 = 3, C3 = 4, T3 = 5, C4 = 6, T4 = 7 };
inline int Cw(int c) { return 2 * (c & 3); }
inline int Tw(int c) { return 2 * (c & 3) + 1; }

// frame m: site at frame position p -> original site index
struct FrameMaps {
    int m[4][4];
    FrameMaps() {
        int cur[4] = {0, 1, 2, 3};
        for (int f = 0; f < 4; ++f) {
            for (int p = 0; p < 4; ++p) m[f][p] = cur[p];
            int nxt[4];
            for (int y = 0; y < 2; ++y)
                for (int x = 0; x < 2; ++x) {
                    const int i = x + 2 * y;
                    const int j = ((2 - y) % 2) + 2 * (x % 2);
                    nxt[j] = cur[i];
                }
            std::memcpy(cur, nxt, sizeof(cur));
        }
    }
    int site(int f, int x, int y) const { return m[f & 3][((x % 2 + 2) % 2) + 2 * ((y % 2 + 2) % 2)]; }
};
const FrameMaps FM;

}  // namespace

struct ctm_ctx {
    std::vector<double> last_spec;  // corner spectra at the previous ctm_spectrum_delta
    std::vector<double> last_loop;  // loop moments at the previous ctm_loop_delta
    int d = 0, D = 0, chi = 0, N = 0, k = 0, q = 0;
    ctm_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    bool have_A[4] = {false, false, false, false};
    unsigned env_set = 0;  // bit (site*8 + which)
    uint64_t rng_counter = 0;
    long long jacobi_capped = 0;  // read_flag calls that saw a capped Jacobi SVD
    int tc_prec = CTM_FP64;       // the tensor-core precision the handle was created with

    std::vector<void*> allocs;
    double* A[4][4] = {};     // [site][rotation]  [s,l,u,r,d]
    double* Alu[4][4] = {};   // [site][rotation]  [l,u,s,r,d]
    double* env[4][8] = {};   // [site][which]
    // scratch
    double *X1 = nullptr, *S1 = nullptr, *S2 = nullptr, *S3 = nullptr;
    double* E[8] = {};        // ul, ur, br, bl of the current cut (E[4..7]: the second cut when batched)
    // second cut's range-finder bases and SVD factors (batch_cuts)
    double *Qm1 = nullptr, *Qb1 = nullptr, *G1 = nullptr, *Us1 = nullptr, *Ws1 = nullptr, *Sv1 = nullptr;
    void* svd2_ws = nullptr;
    double *Pup[2] = {}, *PdnT[2] = {};
    double *Om = nullptr, *Yb = nullptr, *Zb = nullptr, *Qm = nullptr, *Qm2 = nullptr, *Qb = nullptr;
    double *Rb = nullptr, *G = nullptr, *Us = nullptr, *Ws = nullptr, *Sv = nullptr, *inv = nullptr;
    double *Uc = nullptr, *Vc = nullptr, *t1 = nullptr, *t2 = nullptr;
    double *newC1 = nullptr, *newC4 = nullptr, *newT4 = nullptr, *tmpT = nullptr;
    double *Lh = nullptr, *Rh = nullptr, *rho = nullptr, *spec = nullptr, *corners = nullptr;
    double* splitk = nullptr;  // split-K partial sums
    size_t splitk_n = 0;
    // emulated-FP64 tensor-core GEMMs: operand slices and split-K partials
    void *ozA = nullptr, *ozB = nullptr, *ozW = nullptr;
    size_t ozA_n = 0, ozB_n = 0, ozW_n = 0;
    // slices of the four enlarged corners (x plain / transposed), reused by
    // every corner apply of a cut; invalidated by any write to the corner
    struct SliceCache { const double* ptr = nullptr; bool trans = false; void* buf = nullptr; bool valid = false; };
    SliceCache ozc[16];
    // warm start of the range finder: previous sweep's right basis per cut
    double* warmV[16] = {};
    bool warm_valid[16] = {};
    // one warm sweep captured as a CUDA graph and replayed
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool use_graphs = true;
    // optional per-class device timing (ctm_profile_*)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<long long> ev_launch0;  // kernel-launch count at each record's start
    struct Rec { int cls; size_t ev; double flops, bytes; const char* tag; long long launches; };
    std::vector<Rec> recs;
    const char* tag = "other";  // label of the calls being issued (ProfTag)
    struct TagAcc { double ms = 0, flops = 0, bytes = 0; long long calls = 0, launches = 0; };
    std::map<std::string, TagAcc> tags;
    double p_ms[8] = {}, p_flops[8] = {}, p_bytes[8] = {};
    long long p_calls[8] = {};
    void* qr_ws = nullptr;
    void* svd_ws = nullptr;
    void* sval_ws = nullptr;
    unsigned long long* maxbits = nullptr;
    int* flag = nullptr;
    double* dotws = nullptr;   // partial sums of ctm::dot
    double* scal = nullptr;    // scalar results
    // correlation strips (allocated on first use): 9 vectors of chi D^2 chi
    // doubles, 4 ket tensors with an operator applied, 3 d x d operators
    double* cv = nullptr;
    // caller-owned device arena (ctm_create_in): every buffer is carved from
    // it and nothing is freed on destroy
    char* arena = nullptr;
    size_t arena_n = 0, arena_used = 0;
};

namespace {

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            h->err = std::string(#expr) + ": " + cudaGetErrorString(e_);           \
            return CTM_ERR_CUDA;                                                   \
        }                                                                          \
    } while (0)
#define CKS(expr)                           \
    do {                                    \
        ctm_status s_ = (expr);             \
        if (s_ != CTM_OK) return s_;        \
    } while (0)

struct Sizes {
    size_t A, C, T, NN, Nk, Nchi, kk, open;
};

Sizes sizes_of(int d, int D, int chi, int k) {
    Sizes z;
    const size_t N = (size_t)chi * D * D;
    z.A = (size_t)d * D * D * D * D;
    z.C = (size_t)chi * chi;
    z.T = (size_t)chi * D * D * chi;
    z.NN = N * N;
    z.Nk = N * k;
    z.Nchi = N * chi;
    z.kk = (size_t)k * k;
    z.open = (size_t)d * d * N * N;
    return z;
}

int rsvd_k(int N, int chi, const ctm_options& o) {
    if (N <= o.exact_svd_max_n) return N;
    int p = o.rsvd_oversample > 0 ? o.rsvd_oversample : std::max(8, chi / 8);
    return std::min(N, chi + p);
}

// every (M, N, K) a sweep or an RDM contracts (GEMM calls of this file)
std::vector<std::array<long long, 3>> gemm_shapes(int d, int D, int chi, int k) {
    const long long N = (long long)chi * D * D, D2 = (long long)D * D, M3 = (long long)chi * chi * D2;
    return {{chi, N, chi},      {N, N, chi},          {M3, d * D2, D2},     {M3, D2, d * D2},
            {M3 * d, d * D2, D2}, {N, k, N},          {N, chi, k},          {N, chi, N},
            {chi, chi, N},      {chi, N, N},          {N, chi, chi},        {N * D2, chi, chi},
            {(long long)d * d, 1, N * N}, {N * d * d, chi, N}, {(long long)d * d, (long long)d * d, N * chi},
            {k, k, N},          {N, k, k}};
}

// Tensor-core contraction scheme of a precision: -1 FP64 (DFMA), 0 exact-level
// emulated FP64 (CTM_OZAKI_BF16), 1 split-BF16, 2 3xTF32 (both FP32-accumulated)
int tc_mode_of(int precision) {
    switch (precision) {
        case CTM_OZAKI_BF16: return 0;
        case CTM_SPLIT_BF16: return 1;
        case CTM_3XTF32: return 2;
        default: return -1;
    }
}
// operand slices per element of a scheme
int tc_slices_of(const ctm_options& o) {
    switch (tc_mode_of(o.precision)) {
        case 0: return o.ozaki_slices;
        case 1: return 3;
        case 2: return 2;
        default: return 0;
    }
}
size_t tc_split_bytes(int R, int K, int mode, int s) {
    return mode == 2 ? ctm::oz_split_tf32_bytes(R, K) : ctm::oz_split_bytes(R, K, s);
}

struct OzBounds {
    size_t a = 0, b = 0, w = 0;
};
OzBounds oz_bounds(int d, int D, int chi, int k, int s, int mode) {
    OzBounds z;
    for (const auto& sh : gemm_shapes(d, D, chi, k)) {
        z.a = std::max(z.a, tc_split_bytes((int)sh[0], (int)sh[2], mode, s));
        z.b = std::max(z.b, tc_split_bytes((int)sh[1], (int)sh[2], mode, s));
        z.w = std::max(z.w, ctm::oz_gemm_ws_bytes((int)sh[0], (int)sh[1], (int)sh[2], s, mode));
    }
    return z;
}

size_t footprint(int d, int D, const ctm_options& o) {
    const int chi = o.chi;
    const int N = chi * D * D;
    const int k = rsvd_k(N, chi, o);
    Sizes z = sizes_of(d, D, chi, k);
    size_t dbl = 0;
    dbl += 32 * z.A;                 // A, Alu for 4 sites x 4 rotations
    dbl += 16 * z.C + 16 * z.T;      // environments
    dbl += z.T;                      // X1
    dbl += 2 * z.open + (size_t)d * z.NN;  // S1, S3 (open RDM size), S2
    dbl += (o.batch_cuts ? 8 : 4) * z.NN;  // E (both cuts with batch_cuts)
    if (o.batch_cuts) dbl += 2 * z.Nk + 3 * z.kk + (size_t)k;  // second cut's Q, Q_b, G, U', W, S
    dbl += 4 * z.Nchi;               // Pup, PdnT
    dbl += 6 * z.Nk;                 // Om, Y, Z, Qm, Qm2, Qb
    dbl += 4 * z.kk + 2 * (size_t)k; // Rb, G, Us, Ws, Sv, inv
    dbl += z.Nchi + 3 * std::max(z.Nk, z.Nchi);  // Uc; Vc, t1, t2
    dbl += 2 * z.C + 2 * z.T;        // newC1, newC4, newT4, tmpT
    dbl += 2 * z.Nchi * d * d;       // Lh, Rh
    dbl += std::max<size_t>(64 * 64, (size_t)d * d * d * d) + 2 * 16 * z.C;  // rho, spectra, corners
    dbl += (size_t)1 << 24;          // split-K partials
    if (o.rsvd_warm_start && k < N) dbl += 16 * z.Nk;  // warm-start bases
    size_t bytes = dbl * sizeof(double);
    bytes += qr_ws_bytes(N, k) + svd_ws_bytes(k) + svals_ws_bytes(chi, 16);
    if (o.batch_cuts) bytes += svd2_ws_bytes(k);
    bytes += 64 * sizeof(unsigned long long) + 64 + 64 * 256;
    bytes += 256 * 256;  // 256-byte alignment of up to 256 buffers carved from an arena
    bytes += sizeof(double) * (ctm::dot_ws_doubles() + 8);
    const int mode = tc_mode_of(o.precision);
    if (mode >= 0) {
        const int s = tc_slices_of(o);
        const OzBounds z = oz_bounds(d, D, chi, k, s, mode);
        bytes += z.a + z.b + z.w + 3 * 256 + (o.batch_cuts ? 16 : 8) * tc_split_bytes(N, N, mode, s);
    }
    return bytes;
}

ctm_status alloc(ctm_ctx* h, void** p, size_t bytes) {
    if (h->arena) {
        const size_t at = (h->arena_used + 255) & ~(size_t)255, need = bytes ? bytes : 8;
        if (at > h->arena_n || need > h->arena_n - at) {
            h->err = "device arena exhausted";
            return CTM_ERR_OOM;
        }
        *p = h->arena + at;
        h->arena_used = at + need;
        return CTM_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 8);
    if (e != cudaSuccess) {
        h->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return CTM_ERR_OOM;
    }
    h->allocs.push_back(*p);
    return CTM_OK;
}
template <class Tp>
ctm_status allocd(ctm_ctx* h, Tp** p, size_t n) {
    return alloc(h, (void**)p, n * sizeof(Tp));
}
// scratch owned by the caller (cudaFree), for calls that size it per call
template <class Tp>
ctm_status allocd_tmp(ctm_ctx* h, Tp** p, size_t n) {
    if (cudaMalloc((void**)p, (n ? n : 1) * sizeof(Tp)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        h->err = "out of device memory";
        return CTM_ERR_OOM;
    }
    return CTM_OK;
}

// ----------------------------------------------------------------------------
// per-class device timing: an event pair around each call when enabled
// ----------------------------------------------------------------------------
enum { P_GEMM = 0, P_PERM = 1, P_QR = 2, P_SVD = 3, P_SPLIT = 4, P_NCLASS = 8 };
constexpr size_t NO_EV = ~(size_t)0;

size_t prof_begin(ctm_ctx* h) {
    if (!h->prof) return NO_EV;
    while (h->ev_pool.size() < h->ev_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return NO_EV;
        h->ev_pool.push_back(e);
    }
    const size_t i = h->ev_used;
    cudaEventRecord(h->ev_pool[i], h->stream);
    if (h->ev_launch0.size() < h->ev_pool.size()) h->ev_launch0.resize(h->ev_pool.size());
    h->ev_launch0[i] = ctm::g_launches;
    h->ev_used += 2;
    return i;
}
void prof_end(ctm_ctx* h, size_t i, int cls, double flops, double bytes) {
    if (i == NO_EV) return;
    cudaEventRecord(h->ev_pool[i + 1], h->stream);
    h->recs.push_back({cls, i, flops, bytes, h->tag, ctm::g_launches - h->ev_launch0[i]});
}

// labels every profiled call issued in its scope (nested scopes restore)
struct ProfTag {
    ctm_ctx* h;
    const char* prev;
    ProfTag(ctm_ctx* h_, const char* t) : h(h_), prev(h_->tag) {
        static std::mutex mu;
        static std::set<std::string> names;  // interned: records keep the pointer
        std::lock_guard<std::mutex> lock(mu);
        h->tag = names.insert(t).first->c_str();
    }
    ~ProfTag() { h->tag = prev; }
};
void prof_collect(ctm_ctx* h) {
    if (h->recs.empty()) return;
    cudaStreamSynchronize(h->stream);
    for (const auto& r : h->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev_pool[r.ev], h->ev_pool[r.ev + 1]);
        h->p_ms[r.cls] += ms;
        h->p_flops[r.cls] += r.flops;
        h->p_bytes[r.cls] += r.bytes;
        h->p_calls[r.cls] += 1;
        static const char* cls_name[8] = {"gemm", "permute", "qr", "svd", "split", "c5", "c6", "c7"};
        auto& t = h->tags[std::string(r.tag) + "/" + cls_name[r.cls]];
        t.ms += ms;
        t.flops += r.flops;
        t.bytes += r.bytes;
        t.calls += 1;
        t.launches += r.launches;
    }
    h->recs.clear();
    h->ev_used = 0;
}

// ----------------------------------------------------------------------------
// contractions
// ----------------------------------------------------------------------------
// Emulated FP64 product on the tensor cores: s(s+1)/2 BF16 slice products
// of 2 M N K flops each (levels 0..s-1, level L holding L+1 products); its
// algorithmic bytes are the BF16 slices of both operands (K padded to 8) and
// the FP64 output (read too when beta != 0).
double oz_flops(int M, int N, int K, int s) { return 2.0 * M * N * K * (s * (s + 1) / 2); }
double oz_bytes(int M, int N, int K, int s, bool beta, int mode = 0) {
    const double Kp = mode == 2 ? (double)((K + 3) & ~3) : (double)((K + 7) & ~7);
    const double esz = mode == 2 ? 4.0 : 2.0;  // TF32 slices are stored as FP32
    return esz * s * ((double)M * Kp + (double)N * Kp) + 8.0 * M * N * (beta ? 2.0 : 1.0);
}
void slices_written(ctm_ctx* h, const double* p) {
    for (auto& c : h->ozc)
        if (c.ptr == p) c.valid = false;
}
int slice_slot(ctm_ctx* h, const double* A, bool tA, int M, int K) {
    if (!h->ozc[0].buf || M != h->N || K != h->N) return -1;
    for (int c = 0; c < 8; ++c)
        if (A && A == h->E[c]) return 2 * c + (tA ? 1 : 0);
    return -1;
}
// operand slices of the handle's scheme for an R x K operand on strided views
ctm_status split_v(ctm_ctx* h, const double* X, int R, int K, const OzView& rv, const OzView& kv, void* dst) {
    const int mode = tc_mode_of(h->opt.precision), s = tc_slices_of(h->opt);
    const size_t ev = prof_begin(h);
    if (mode == 2) CK(ctm::oz_split_tf32(X, R, K, rv, kv, dst, h->stream));
    else CK(ctm::oz_split_view(X, R, K, rv, kv, s, dst, h->stream));
    prof_end(h, ev, P_SPLIT, 0.0, (8.0 + (mode == 2 ? 8.0 : 2.0 * s)) * (double)R * K);
    return CTM_OK;
}
ctm_status split_(ctm_ctx* h, const double* X, int R, int K, long long rs, long long cs, void* dst) {
    if (tc_mode_of(h->opt.precision) == 2) {
        const OzView rv{1, {R, 1, 1, 1}, {rs, 0, 0, 0}}, kv{1, {K, 1, 1, 1}, {cs, 0, 0, 0}};
        return split_v(h, X, R, K, rv, kv, dst);
    }
    const size_t ev = prof_begin(h);
    CK(ctm::oz_split(X, R, K, rs, cs, tc_slices_of(h->opt), dst, h->stream));
    prof_end(h, ev, P_SPLIT, 0.0, (8.0 + 2.0 * tc_slices_of(h->opt)) * (double)R * K);
    return CTM_OK;
}

ctm_status gemm(ctm_ctx* h, bool tA, bool tB, int M, int N, int K, const double* A, int lda,
                const double* B, int ldb, double* C, int ldc, double beta = 0.0) {
    slices_written(h, C);
    const double flops = 2.0 * M * N * K;
    const double bytes = 8.0 * ((double)M * K + (double)K * N + (double)M * N);
    // a matrix-vector product gains nothing from 128-wide tensor tiles
    const int mode = tc_mode_of(h->opt.precision);
    if (mode >= 0 && M > 0 && N > 1 && K > 0) {
        const int s = tc_slices_of(h->opt);
        if (tc_split_bytes(M, K, mode, s) > h->ozA_n || tc_split_bytes(N, K, mode, s) > h->ozB_n ||
            ctm::oz_gemm_ws_bytes(M, N, K, s, mode) > h->ozW_n) {
            h->err = "emulated GEMM: shape outside the handle's workspace";
            return CTM_ERR_STATE;
        }
        // op(A)[m][k] and op(B)[k][n] as row views of M x K and N x K
        const int slot = slice_slot(h, A, tA, M, K);
        void* sa = slot >= 0 ? h->ozc[slot].buf : h->ozA;
        if (slot < 0 || !h->ozc[slot].valid) {
            CKS(split_(h, A, M, K, tA ? 1 : lda, tA ? lda : 1, sa));
            if (slot >= 0) h->ozc[slot].valid = true;
        }
        CKS(split_(h, B, N, K, tB ? ldb : 1, tB ? 1 : ldb, h->ozB));
        const size_t ev = prof_begin(h);
        CK(ctm::oz_gemm(M, N, K, s, sa, h->ozB, 1.0, beta, C, ldc, h->ozW, h->ozW_n, h->flag + 1, h->stream,
                        mode));
        prof_end(h, ev, P_GEMM, oz_flops(M, N, K, s), oz_bytes(M, N, K, s, beta != 0.0, mode));
    } else {
        const size_t ev = prof_begin(h);
        CK(ctm::dgemm(tA, tB, M, N, K, 1.0, A, lda, B, ldb, beta, C, ldc, h->stream, h->splitk, h->splitk_n));
        prof_end(h, ev, P_GEMM, flops, bytes);
    }
    return CTM_OK;
}
// emulated GEMM on strided views: op(A) element (m, k) at A[view(ar, m) +
// view(ak, k)], op(B) element (k, n) at B[view(bn, n) + view(bk, k)], C
// element (m, n) written at C[view(cr, m) + view(cc, n)]
ctm_status gemm_v(ctm_ctx* h, int M, int N, int K, const double* A, const OzView& ar, const OzView& ak,
                  const double* B, const OzView& bn, const OzView& bk, double* C, const OzView& cr,
                  const OzView& cc) {
    slices_written(h, C);
    const int mode = tc_mode_of(h->opt.precision), s = tc_slices_of(h->opt);
    if (tc_split_bytes(M, K, mode, s) > h->ozA_n || tc_split_bytes(N, K, mode, s) > h->ozB_n ||
        ctm::oz_gemm_ws_bytes(M, N, K, s, mode) > h->ozW_n) {
        h->err = "emulated GEMM: shape outside the handle's workspace";
        return CTM_ERR_STATE;
    }
    CKS(split_v(h, A, M, K, ar, ak, h->ozA));
    CKS(split_v(h, B, N, K, bn, bk, h->ozB));
    const size_t ev = prof_begin(h);
    CK(ctm::oz_gemm_view(M, N, K, s, h->ozA, h->ozB, 1.0, 0.0, C, cr, cc, h->ozW, h->ozW_n, h->flag + 1,
                         h->stream, mode));
    prof_end(h, ev, P_GEMM, oz_flops(M, N, K, s), oz_bytes(M, N, K, s, false, mode));
    return CTM_OK;
}

ctm_status perm(ctm_ctx* h, const double* src, double* dst, std::initializer_list<int> dims,
                std::initializer_list<int> p) {
    std::vector<int> dv(dims), pv(p);
    double n = 1;
    for (int v : dv) n *= v;
    slices_written(h, dst);
    const size_t ev = prof_begin(h);
    CK(ctm::permute(src, dst, (int)dv.size(), dv.data(), pv.data(), h->stream));
    prof_end(h, ev, P_PERM, 0.0, 16.0 * n);
    return CTM_OK;
}
ctm_status qr_(ctm_ctx* h, const double* Y, double* Q, double* R) {
    ProfTag tg(h, "qr");
    const size_t ev = prof_begin(h);
    CK(ctm::qr(Y, h->N, h->k, Q, R, h->qr_ws, h->stream, h->flag + 1));
    prof_end(h, ev, P_QR, 4.0 * h->N * (double)h->k * h->k, 0.0);
    return CTM_OK;
}
ctm_status svd_(ctm_ctx* h) {
    ProfTag tg(h, "svd");
    const size_t ev = prof_begin(h);
    CK(ctm::svd(h->G, h->k, h->Us, h->Sv, h->Ws, h->svd_ws, h->stream, h->flag + 2));
    prof_end(h, ev, P_SVD, 0.0, 0.0);
    return CTM_OK;
}

// X1[g,u,u',b] (chi x D x D x chi), Tp[a,l,l',g], A / Alu of one rotation.
// closed: out[(a,d,d'), (b,r,r')] (N x N).
// open:   out[a,b,r,d,s,t,r',d'] (d^2 N^2), physical indices left open.
ctm_status corner_core(ctm_ctx* h, const double* X1, const double* Tp, const double* A,
                       const double* Alu, double* out, bool open) {
    const int chi = h->chi, D = h->D, d = h->d, N = h->N;
    const int D2 = D * D;
    const char* outer = h->tag;
    const std::string t2 = std::string(outer) + ".X2", t3 = std::string(outer) + ".X3",
                      t4 = std::string(outer) + ".X4";
    if (tc_mode_of(h->opt.precision) >= 0 && !open) {
        // Tensor-core path.  Every permutation is folded into operand views and
        // output layouts, chosen so that both large intermediates are plain
        // K-contiguous row matrices (single-pass slicing) and the epilogue
        // writes of X2 and X3 run along contiguous memory:
        //   S1[a][b][l'][u'][l][u] = X2,  S2[a][b][r][d][s][l'][u'] = X3.
        const long long c = chi, Dl = D, dD2 = (long long)d * D2, D4 = (long long)D2 * D2, M3 = c * c * D2;
        {
            // X2^T[(b,u',u), (a,l,l')] = sum_g X1[g,u,u',b] Tp[a,l,l',g]
            ProfTag tg(h, t2.c_str());
            const OzView x1r{3, {chi, D, D, 1}, {1, c, Dl * c, 0}}, x1k{1, {chi, 1, 1, 1}, {N, 0, 0, 0}};
            const OzView tpn{1, {N, 1, 1, 1}, {c, 0, 0, 0}}, tpk{1, {chi, 1, 1, 1}, {1, 0, 0, 0}};
            const OzView s1r{3, {chi, D, D, 1}, {D4, D2, 1, 0}}, s1c{3, {chi, D, D, 1}, {c * D4, Dl, Dl * D2, 0}};
            CKS(gemm_v(h, N, N, chi, X1, x1r, x1k, Tp, tpn, tpk, h->S1, s1r, s1c));
        }
        {
            // X3[(a,b,l',u'), (s,r,d)] = S1[(a,b,l',u'), (l,u)] Alu[(l,u), (s,r,d)]
            ProfTag tg(h, t3.c_str());
            const OzView x2r{1, {(int)M3, 1, 1, 1}, {D2, 0, 0, 0}}, x2k{1, {D2, 1, 1, 1}, {1, 0, 0, 0}};
            const OzView alu_n{1, {(int)dD2, 1, 1, 1}, {1, 0, 0, 0}}, alu_k{1, {D2, 1, 1, 1}, {dD2, 0, 0, 0}};
            const OzView x3r{3, {chi * chi, D, D, 1}, {D2 * dD2, Dl, 1, 0}};
            const OzView x3c{3, {d, D, D, 1}, {D2, Dl * dD2, dD2, 0}};
            CKS(gemm_v(h, (int)M3, (int)dD2, D2, h->S1, x2r, x2k, Alu, alu_n, alu_k, h->S2, x3r, x3c));
        }
        // E[(a,d,d'), (b,r,r')] = S2[(a,b,r,d), (s,l',u')] A[(s,l',u'), (r',d')]
        const OzView s2r{1, {(int)M3, 1, 1, 1}, {dD2, 0, 0, 0}}, s2k{1, {(int)dD2, 1, 1, 1}, {1, 0, 0, 0}};
        const OzView a_n{1, {D2, 1, 1, 1}, {1, 0, 0, 0}}, a_k{1, {(int)dD2, 1, 1, 1}, {D2, 0, 0, 0}};
        const OzView qr{4, {chi, chi, D, D}, {(long long)D2 * N, D2, Dl, Dl * N}};
        const OzView qc{2, {D, D, 1, 1}, {1, N, 0, 0}};
        ProfTag tg(h, t4.c_str());
        return gemm_v(h, (int)M3, D2, (int)dD2, h->S2, s2r, s2k, A, a_n, a_k, out, qr, qc);
    }
    // X2[(a,l,l'), (u,u',b)] = Tp[(a,l,l'), g] X1[g, (u,u',b)]
    {
        ProfTag tg(h, t2.c_str());
        CKS(gemm(h, false, false, N, N, chi, Tp, chi, X1, N, h->S1, N));
    }
    // -> [a,l',u',b,l,u]
    CKS(perm(h, h->S1, h->S2, {chi, D, D, D, D, chi}, {0, 2, 4, 5, 1, 3}));
    // X3[(a,l',u',b), (s,r,d)] = X2p[(a,l',u',b), (l,u)] Alu[(l,u), (s,r,d)]
    const int M3 = chi * chi * D2;
    CKS(gemm(h, false, false, M3, d * D2, D2, h->S2, D2, Alu, d * D2, h->S1, d * D2));
    // -> [a,b,r,d,s,l',u']
    CKS(perm(h, h->S1, h->S2, {chi, D, D, chi, d, D, D}, {0, 3, 5, 6, 4, 1, 2}));
    if (!open) {
        // X4[(a,b,r,d), (r',d')] = X3p[(a,b,r,d), (s,l',u')] A[(s,l',u'), (r',d')]
        CKS(gemm(h, false, false, M3, D2, d * D2, h->S2, d * D2, A, D2, h->S1, D2));
        // -> [a,d,d',b,r,r']
        CKS(perm(h, h->S1, out, {chi, chi, D, D, D, D}, {0, 3, 5, 1, 2, 4}));
    } else {
        // X4o[(a,b,r,d,s), (t,r',d')] = X3p[(a,b,r,d,s), (l',u')] Alu[(l',u'), (t,r',d')]
        CKS(gemm(h, false, false, M3 * d, d * D2, D2, h->S2, D2, Alu, d * D2, out, d * D2));
    }
    return CTM_OK;
}

// corner c (0..3 = C1..C4 position) of site i as an N x N matrix.
ctm_status enlarged_corner(ctm_ctx* h, int i, int c, double* out) {
    ProfTag tg(h, "corner");
    const int chi = h->chi, N = h->N;
    CKS(gemm(h, false, false, chi, N, chi, h->env[i][Cw(c)], chi, h->env[i][Tw(c)], N, h->X1, N));
    return corner_core(h, h->X1, h->env[i][Tw(c + 3)], h->A[i][c & 3], h->Alu[i][c & 3], out, false);
}

// ----------------------------------------------------------------------------
// randomised SVD of M = H_u^T H_d and the projectors of one cut
// ----------------------------------------------------------------------------
// E: the four enlarged corners ul, ur, br, bl of the cut
ctm_status applyM(ctm_ctx* h, double* const* E, const double* X, double* out, int cols) {
    ProfTag tg(h, "rsvd.apply");
    const int N = h->N;
    CKS(gemm(h, true, false, N, cols, N, E[2], N, X, cols, h->t1, cols));      // E_br^T X
    CKS(gemm(h, true, false, N, cols, N, E[3], N, h->t1, cols, h->t2, cols));  // E_bl^T
    CKS(gemm(h, true, false, N, cols, N, E[0], N, h->t2, cols, h->t1, cols));  // E_ul^T
    CKS(gemm(h, true, false, N, cols, N, E[1], N, h->t1, cols, out, cols));    // E_ur^T
    return CTM_OK;
}
ctm_status applyMT(ctm_ctx* h, double* const* E, const double* X, double* out, int cols) {
    ProfTag tg(h, "rsvd.apply");
    const int N = h->N;
    CKS(gemm(h, false, false, N, cols, N, E[1], N, X, cols, h->t1, cols));      // E_ur X
    CKS(gemm(h, false, false, N, cols, N, E[0], N, h->t1, cols, h->t2, cols));  // E_ul
    CKS(gemm(h, false, false, N, cols, N, E[3], N, h->t2, cols, h->t1, cols));  // E_bl
    CKS(gemm(h, false, false, N, cols, N, E[2], N, h->t1, cols, out, cols));    // E_br
    return CTM_OK;
}

// what one cut keeps from its range finder to its projectors
struct CutBufs {
    double* const* E;
    double *Qm, *Qb, *G, *Us, *Ws, *Sv;
};
CutBufs cut_bufs(ctm_ctx* h, int which) {
    if (which == 0) return CutBufs{h->E, h->Qm, h->Qb, h->G, h->Us, h->Ws, h->Sv};
    return CutBufs{h->E + 4, h->Qm1, h->Qb1, h->G1, h->Us1, h->Ws1, h->Sv1};
}

// cut: (frame, column, row) index 0..15, keys the warm-start basis.
// Range finder of M = H_u^T H_d up to the small factor G = R_b^T.
ctm_status range_finder(ctm_ctx* h, int cut, const CutBufs& c) {
    ProfTag tg(h, "projector");
    const int N = h->N, k = h->k;
    const bool warm_on = h->opt.rsvd_warm_start && k < N;
    const bool warm = warm_on && h->warm_valid[cut];
    const int q = (k == N || warm) ? 0 : h->q;
    const double* Om = h->Om;
    if (warm) Om = h->warmV[cut];  // one more subspace iteration from last sweep's basis
    else CK(ctm::rng_normal(h->Om, (size_t)N * k, h->opt.seed, h->rng_counter++, h->stream));
    CKS(applyM(h, c.E, Om, h->Yb, k));
    // Householder QR for every basis: a Gram-based (Cholesky) QR resolves
    // only directions above ~1e-8 of the largest, while the 1e-12 cutoff keeps
    // directions down to 1e-12; with a warm basis that lags a still-changing
    // environment that loss stopped the D=8, chi=128 iteration converging.
    CKS(qr_(h, h->Yb, c.Qm, h->Rb));
    for (int it = 0; it < q; ++it) {
        CKS(applyMT(h, c.E, c.Qm, h->Zb, k));
        CKS(qr_(h, h->Zb, h->Qm2, h->Rb));
        CKS(applyM(h, c.E, h->Qm2, h->Yb, k));
        CKS(qr_(h, h->Yb, c.Qm, h->Rb));
    }
    // B^T = M^T Q = Q_b R_b  ->  B = R_b^T Q_b^T ; SVD(R_b^T) = U' S W^T
    CKS(applyMT(h, c.E, c.Qm, h->Zb, k));
    CKS(qr_(h, h->Zb, c.Qb, h->Rb));
    return perm(h, h->Rb, c.G, {k, k}, {1, 0});
}

// Projectors of a cut from the SVD of its small factor.
ctm_status finish_projectors(ctm_ctx* h, int slot, int cut, const CutBufs& c) {
    ProfTag tg(h, "projector");
    const int N = h->N, k = h->k, chi = h->chi;
    const bool warm_on = h->opt.rsvd_warm_start && k < N;
    // U = Q U'[:, :chi].  V = Q_b W over all k columns, sorted by singular
    // value: its first chi columns are the projector's V, and the whole basis
    // (the span of Q_b) starts this cut's range finder in the next sweep,
    // where it leaves R_b close to diagonal once the environment settles, so
    // that the Jacobi SVD starts near its quadratic phase.
    double* Vf = warm_on ? h->warmV[cut] : h->Vc;
    CKS(gemm(h, false, false, N, chi, k, c.Qm, k, c.Us, k, h->Uc, chi));
    CKS(gemm(h, false, false, N, k, k, c.Qb, k, c.Ws, k, Vf, k));
    if (warm_on) h->warm_valid[cut] = true;
    CK(ctm::inv_sqrt_cut(c.Sv, h->inv, chi, h->opt.sv_cutoff_rel, h->stream));
    // P_up = E_bl^T (E_br^T V) S^-1/2 ; P_dn^T = E_ul (E_ur U) S^-1/2
    CKS(gemm(h, true, false, N, chi, N, c.E[2], N, Vf, k, h->t1, chi));
    CKS(gemm(h, true, false, N, chi, N, c.E[3], N, h->t1, chi, h->Pup[slot], chi));
    CK(ctm::scale_cols(h->Pup[slot], N, chi, chi, h->inv, h->stream));
    CKS(gemm(h, false, false, N, chi, N, c.E[1], N, h->Uc, chi, h->t1, chi));
    CKS(gemm(h, false, false, N, chi, N, c.E[0], N, h->t1, chi, h->PdnT[slot], chi));
    CK(ctm::scale_cols(h->PdnT[slot], N, chi, chi, h->inv, h->stream));
    return CTM_OK;
}

ctm_status projectors(ctm_ctx* h, int slot, int cut) {
    const CutBufs c = cut_bufs(h, 0);
    CKS(range_finder(h, cut, c));
    CKS(svd_(h));
    return finish_projectors(h, slot, cut, c);
}

// both cuts' SVDs in one launch (two Jacobi clusters)
ctm_status svd2_(ctm_ctx* h, const CutBufs& a, const CutBufs& b) {
    ProfTag tg(h, "svd");
    const size_t ev = prof_begin(h);
    CK(ctm::svd2(a.G, b.G, h->k, a.Us, a.Sv, a.Ws, b.Us, b.Sv, b.Ws, h->svd2_ws, h->stream, h->flag + 2));
    prof_end(h, ev, P_SVD, 0.0, 0.0);
    return CTM_OK;
}

ctm_status normalise_into(ctm_ctx* h, const double* src, double* dst, size_t n, int slot) {
    CK(cudaMemsetAsync(h->maxbits + slot, 0, sizeof(unsigned long long), h->stream));
    CK(ctm::maxabs(src, n, h->maxbits + slot, h->stream));
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CK(ctm::scale_by_max(dst, n, h->maxbits + slot, h->flag, h->stream));
    return CTM_OK;
}

// absorb column x of frame m into the left boundary of column x+1
ctm_status left_move(ctm_ctx* h, int m, int x) {
    const int chi = h->chi, N = h->N, D = h->D;
    const bool both = h->E[4] != nullptr;  // batch_cuts: corners of both cuts resident
    for (int y = 0; y < 2; ++y) {
        const int tl = FM.site(m, x, y + 1), tr = FM.site(m, x + 1, y + 1);
        const int br = FM.site(m, x + 1, y), bl = FM.site(m, x, y);
        double* const* E = both ? h->E + 4 * y : h->E;
        CKS(enlarged_corner(h, tl, m + 0, E[0]));
        CKS(enlarged_corner(h, tr, m + 1, E[1]));
        CKS(enlarged_corner(h, br, m + 2, E[2]));
        CKS(enlarged_corner(h, bl, m + 3, E[3]));
        const int cut = ((m & 3) * 2 + x) * 2 + y;
        if (!both) CKS(projectors(h, y, cut));
        else CKS(range_finder(h, cut, cut_bufs(h, y)));
    }
    if (both) {
        CKS(svd2_(h, cut_bufs(h, 0), cut_bufs(h, 1)));
        for (int y = 0; y < 2; ++y) CKS(finish_projectors(h, y, ((m & 3) * 2 + x) * 2 + y, cut_bufs(h, y)));
    }
    ProfTag tg(h, "absorb");
    for (int y = 0; y < 2; ++y) {
        const int i = FM.site(m, x, y), j = FM.site(m, x + 1, y);
        const int ym = (y + 1) % 2;  // cut between rows y-1 and y
        double** e = h->env[i];
        // C1' = P_up(y)^T (C1 T1)
        CKS(gemm(h, false, false, chi, N, chi, e[Cw(m)], chi, e[Tw(m)], N, h->X1, N));
        CKS(gemm(h, true, false, chi, chi, N, h->Pup[y], chi, h->X1, chi, h->newC1, chi));
        // T4' = P_up(y-1)^T core(P_dn(y)^T, T4, A)   -> [c1, c2, r, r'] -> [c1, r, r', c2]
        CKS(corner_core(h, h->PdnT[y], e[Tw(m + 3)], h->A[i][m & 3], h->Alu[i][m & 3], h->E[0], false));
        CKS(gemm(h, true, false, chi, N, N, h->Pup[ym], chi, h->E[0], N, h->tmpT, N));
        CKS(perm(h, h->tmpT, h->newT4, {chi, chi, D, D}, {0, 2, 3, 1}));
        // C4' = (C4 T3)^T P_dn(y-1)^T :  Z[z,d,d',g] = T3[(z,d,d'),h] C4[h,g] -> [z,g,d,d']
        CKS(gemm(h, false, false, N, chi, chi, e[Tw(m + 2)], chi, e[Cw(m + 3)], chi, h->t1, chi));
        CKS(perm(h, h->t1, h->t2, {chi, D, D, chi}, {0, 3, 1, 2}));
        CKS(gemm(h, false, false, chi, chi, N, h->t2, N, h->PdnT[ym], chi, h->newC4, chi));
        double** ej = h->env[j];
        CKS(normalise_into(h, h->newC1, ej[Cw(m)], (size_t)chi * chi, 0));
        CKS(normalise_into(h, h->newT4, ej[Tw(m + 3)], (size_t)chi * N, 1));
        CKS(normalise_into(h, h->newC4, ej[Cw(m + 3)], (size_t)chi * chi, 2));
    }
    return CTM_OK;
}

ctm_status one_sweep_eager(ctm_ctx* h) {
    for (int m = 0; m < 4; ++m)
        for (int x = 0; x < 2; ++x) CKS(left_move(h, m, x));
    return CTM_OK;
}

// A sweep's launch sequence is fixed once every cut has a warm basis (or
// when the range finder never warm-starts): capture it once, replay it.
ctm_status one_sweep(ctm_ctx* h) {
    bool steady = !h->opt.rsvd_warm_start || h->k == h->N;
    if (!steady) {
        steady = true;
        for (bool w : h->warm_valid) steady = steady && w;
    }
    if (!h->use_graphs || h->prof || !steady) return one_sweep_eager(h);
    if (!h->graph_exec) {
        CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const ctm_status st = one_sweep_eager(h);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (st != CTM_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        CK(e);
        h->graph = g;
        CK(cudaGraphInstantiate(&h->graph_exec, h->graph, 0));
    }
    CK(cudaGraphLaunch(h->graph_exec, h->stream));
    return CTM_OK;
}

// Switches the handle's contractions between emulated FP64 and FP64 (every
// buffer either needs exists from ctm_create on); the captured sweep graph
// is dropped, the range finder's warm bases are kept.
// Where the loop-moment change of a scheme stalls (measured at d=2, D=6,
// chi=72): FP32-summed split-BF16 / 3xTF32 near 1e-5, emulated FP64 with 3
// slices near 1e-6, 4 slices near 2e-8, 5 and more below 1e-9.  fp64_refine
// hands over to FP64 a decade above the stall.
double refine_at(const ctm_options& o) {
    switch (tc_mode_of(o.precision)) {
        case 0: return o.ozaki_slices >= 5 ? 1e-8 : o.ozaki_slices == 4 ? 2e-7 : 1e-5;
        case 1:
        case 2: return 1e-4;
        default: return 0.0;
    }
}
ctm_status set_precision(ctm_ctx* h, int precision) {
    if (h->opt.precision == precision) return CTM_OK;
    if (precision != CTM_FP64 && precision != h->tc_prec) {
        h->err = "a handle switches only between FP64 and the tensor-core precision it was created with";
        return CTM_ERR_STATE;
    }
    CK(cudaStreamSynchronize(h->stream));
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph_exec = nullptr;
    h->graph = nullptr;
    for (auto& c : h->ozc) c.valid = false;
    h->opt.precision = precision;
    return CTM_OK;
}

ctm_status check_ready(ctm_ctx* h) {
    for (int i = 0; i < 4; ++i)
        if (!h->have_A[i]) {
            h->err = "site tensors not set";
            return CTM_ERR_STATE;
        }
    if (h->env_set != 0xffffffffu) {
        h->err = "environment not set (all 8 tensors of all 4 sites)";
        return CTM_ERR_STATE;
    }
    return CTM_OK;
}

ctm_status read_flag(ctm_ctx* h) {
    int f[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(f, h->flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (f[2]) {  // a projector SVD hit the Jacobi sweep cap: counted, not an error
        ++h->jacobi_capped;
        CK(cudaMemsetAsync(h->flag + 2, 0, sizeof(int), h->stream));
    }
    if (f[1]) {
        h->err = "a bounded device wait (tensor-core GEMM pipeline or QR grid barrier) gave up";
        return CTM_ERR_TIMEOUT;
    }
    if (f[0] == 2) {
        h->err = "an environment tensor became zero (every projector direction was cut)";
        return CTM_ERR_NONFINITE;
    }
    if (f[0]) {
        h->err = "non-finite environment";
        return CTM_ERR_NONFINITE;
    }
    return CTM_OK;
}

ctm_status spectra(ctm_ctx* h, std::vector<double>& out) {
    const int chi = h->chi;
    const size_t C = (size_t)chi * chi;
    for (int i = 0; i < 4; ++i)
        for (int c = 0; c < 4; ++c)
            CK(cudaMemcpyAsync(h->corners + (i * 4 + c) * C, h->env[i][Cw(c)], C * sizeof(double),
                               cudaMemcpyDeviceToDevice, h->stream));
    CK(ctm::svals_normalised(h->corners, chi, 16, h->spec, h->sval_ws, h->stream));
    out.resize(16 * (size_t)chi);
    CK(cudaMemcpyAsync(out.data(), h->spec, out.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return CTM_OK;
}

// Gauge-invariant convergence measure: for the 2x2 block with bottom-left
// site i, the corner loop L = C1(TL) C2(TR) C3(BR) C4(BL) (the network Z_00)
// changes under a change of basis G on any chi bond only to a similar
// matrix, so the normalised moments m_p = Tr(L^p) / Tr(L)^p, p = 2, 3, 4 (sums
// of the p-th powers of the loop eigenvalues normalised to sum 1) do not
// depend on the gauge the projectors leave on the chi bonds, while the
// singular values of a single corner do.  The moments are also unchanged by
// L -> c L, so the free overall sign each corner carries (every C is divided
// by its own largest |entry|) drops out.  FP64 products (chi^3 each).
// out: 4 blocks x 3 moments; NaN where Tr(L) is zero or not finite.
ctm_status loop_moments(ctm_ctx* h, std::vector<double>& out) {
    const int chi = h->chi;
    const size_t C = (size_t)chi * chi;
    double* w = h->corners;  // 16 chi^2 scratch: ta, tb, L, L2, L3, L4 per block in turn
    double* ta = w;
    double* tb = w + C;
    double* L = w + 2 * C;  // L, L^2, L^3, L^4 contiguous for one traces() call
    double tr[16];
    out.assign(12, 0.0);
    for (int i = 0; i < 4; ++i) {
        const int x = i % 2, y = i / 2;
        auto site = [](int xx, int yy) { return ((xx % 2 + 2) % 2) + 2 * ((yy % 2 + 2) % 2); };
        const double* c1 = h->env[site(x, y + 1)][C1];
        const double* c2 = h->env[site(x + 1, y + 1)][C2];
        const double* c3 = h->env[site(x + 1, y)][C3];
        const double* c4 = h->env[site(x, y)][C4];
        CK(ctm::dgemm(false, false, chi, chi, chi, 1.0, c1, chi, c2, chi, 0.0, ta, chi, h->stream));
        CK(ctm::dgemm(false, false, chi, chi, chi, 1.0, ta, chi, c3, chi, 0.0, tb, chi, h->stream));
        CK(ctm::dgemm(false, false, chi, chi, chi, 1.0, tb, chi, c4, chi, 0.0, L, chi, h->stream));
        CK(ctm::dgemm(false, false, chi, chi, chi, 1.0, L, chi, L, chi, 0.0, L + C, chi, h->stream));
        CK(ctm::dgemm(false, false, chi, chi, chi, 1.0, L + C, chi, L, chi, 0.0, L + 2 * C, chi, h->stream));
        CK(ctm::dgemm(false, false, chi, chi, chi, 1.0, L + C, chi, L + C, chi, 0.0, L + 3 * C, chi, h->stream));
        CK(ctm::traces(L, chi, 4, h->scal + 4 * (i % 2), h->stream));
        if (i % 2 == 1 || i == 3) {
            CK(cudaMemcpyAsync(tr + 4 * (i - 1), h->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
    }
    for (int i = 0; i < 4; ++i) {
        const double t1 = tr[4 * i];
        for (int p = 2; p <= 4; ++p)
            out[3 * i + (p - 2)] = (t1 != 0.0 && std::isfinite(t1)) ? tr[4 * i + p - 1] / std::pow(t1, (double)p)
                                                                   : NAN;
    }
    return CTM_OK;
}

// ----------------------------------------------------------------------------
// reduced density matrices
// ----------------------------------------------------------------------------
ctm_status rdm1_dev(ctm_ctx* h, int i, std::vector<double>& rho) {
    const int chi = h->chi, D = h->D, d = h->d, N = h->N;
    double** e = h->env[i];
    CKS(gemm(h, false, false, chi, N, chi, e[C1], chi, e[T1], N, h->X1, N));
    CKS(corner_core(h, h->X1, e[T4], h->A[i][0], h->Alu[i][0], h->S3, true));  // [a,b,r,d,s,t,r',d']
    // ring C2 T2 C3 T3 C4 -> [b,r,r',d,d',a]
    CKS(gemm(h, false, false, chi, N, chi, e[C2], chi, e[T2], N, h->t1, N));          // [b,r,r',e]
    CKS(gemm(h, false, false, N, chi, chi, h->t1, chi, e[C3], chi, h->t2, chi));      // [b,r,r',f]
    CKS(gemm(h, false, false, N, N, chi, h->t2, chi, e[T3], N, h->E[0], N));          // [b,r,r',d,d',g]
    CKS(gemm(h, false, false, N * D * D, chi, chi, h->E[0], chi, e[C4], chi, h->E[1], chi));  // [..,a]
    CKS(perm(h, h->E[1], h->E[2], {chi, D, D, D, D, chi}, {5, 0, 1, 3, 2, 4}));      // [a,b,r,d,r',d']
    CKS(perm(h, h->S3, h->S1, {chi, chi, D, D, d, d, D, D}, {4, 5, 0, 1, 2, 3, 6, 7}));  // [s,t,...]
    CKS(gemm(h, false, false, d * d, 1, N * N, h->S1, N * N, h->E[2], 1, h->rho, 1));
    rho.resize((size_t)d * d);
    CK(cudaMemcpyAsync(rho.data(), h->rho, rho.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return CTM_OK;
}

// horizontal pair in frame f: L at frame (x,y), R at frame (x+1,y); rho over (L, R)
ctm_status rdm2_h_dev(ctm_ctx* h, int f, int L, int R, std::vector<double>& out) {
    const int chi = h->chi, D = h->D, d = h->d, N = h->N;
    double** eL = h->env[L];
    double** eR = h->env[R];
    const int c0 = f & 3, c1 = (f + 1) & 3;
    // left half: E_ul(L) open, contracted with C4 T3 of L over its down leg
    CKS(gemm(h, false, false, chi, N, chi, eL[Cw(c0)], chi, eL[Tw(c0)], N, h->X1, N));
    CKS(corner_core(h, h->X1, eL[Tw(c0 + 3)], h->A[L][c0], h->Alu[L][c0], h->S3, true));
    CKS(perm(h, h->S3, h->S1, {chi, chi, D, D, d, d, D, D}, {1, 2, 6, 4, 5, 0, 3, 7}));  // [b,r,r',s,t,a,d,d']
    CKS(gemm(h, false, false, N, chi, chi, eL[Tw(c0 + 2)], chi, eL[Cw(c0 + 3)], chi, h->t1, chi));  // [z,d,d',g]
    CKS(perm(h, h->t1, h->t2, {chi, D, D, chi}, {3, 1, 2, 0}));                       // [g,d,d',z]
    CKS(gemm(h, false, false, N * d * d, chi, N, h->S1, N, h->t2, chi, h->Lh, chi));   // [b,r,r',s,t,k]
    // right half: E_ur(R) open (rows = left leg, cols = down leg), cols contracted with C3 T3 of R
    CKS(gemm(h, false, false, chi, N, chi, eR[Cw(c1)], chi, eR[Tw(c1)], N, h->X1, N));
    CKS(corner_core(h, h->X1, eR[Tw(c1 + 3)], h->A[R][c1], h->Alu[R][c1], h->S3, true));
    CKS(perm(h, h->S3, h->S1, {chi, chi, D, D, d, d, D, D}, {0, 3, 7, 4, 5, 1, 2, 6}));  // [a,d,d',s,t,b,r,r']
    CKS(gemm(h, false, false, chi, N, chi, eR[Cw(c0 + 2)], chi, eR[Tw(c0 + 2)], N, h->t1, N));  // [b,d,d',k]
    CKS(gemm(h, false, false, N * d * d, chi, N, h->S1, N, h->t1, chi, h->Rh, chi));   // [a,d,d',s,t,k]
    // contract over (chi, D, D, chi): [p,q | b,r,r',k] x [s,t | b,r,r',k]
    CKS(perm(h, h->Lh, h->S1, {chi, D, D, d, d, chi}, {3, 4, 0, 1, 2, 5}));
    CKS(perm(h, h->Rh, h->S3, {chi, D, D, d, d, chi}, {3, 4, 0, 1, 2, 5}));
    CKS(gemm(h, false, true, d * d, d * d, N * chi, h->S1, N * chi, h->S3, N * chi, h->rho, d * d));
    std::vector<double> r((size_t)d * d * d * d);
    CK(cudaMemcpyAsync(r.data(), h->rho, r.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // r[p,q,s,t] (p,q = ket,bra of L; s,t = ket,bra of R) -> rho[(p,s),(q,t)]
    out.assign(r.size(), 0.0);
    for (int p = 0; p < d; ++p)
        for (int qq = 0; qq < d; ++qq)
            for (int s = 0; s < d; ++s)
                for (int t = 0; t < d; ++t)
                    out[((size_t)(p * d + s)) * d * d + (qq * d + t)] = r[((p * d + qq) * d + s) * d + t];
    return CTM_OK;
}

void normalise_trace(std::vector<double>& rho, int n) {
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += rho[(size_t)i * n + i];
    if (tr != 0.0)
        for (double& v : rho) v /= tr;
}

ctm_status rdm2_any(ctm_ctx* h, int site, int dx, int dy, std::vector<double>& rho) {
    const int d = h->d;
    const int x = site % 2, y = site / 2;
    const int j = ((x + dx) % 2 + 2) % 2 + 2 * (((y + dy) % 2 + 2) % 2);
    std::vector<double> r;
    bool swap = false;
    if (dx == 1 && dy == 0) { CKS(rdm2_h_dev(h, 0, site, j, r)); }
    else if (dx == -1 && dy == 0) { CKS(rdm2_h_dev(h, 0, j, site, r)); swap = true; }
    else if (dx == 0 && dy == 1) { CKS(rdm2_h_dev(h, 1, j, site, r)); swap = true; }   // frame 1: top site is left
    else if (dx == 0 && dy == -1) { CKS(rdm2_h_dev(h, 1, site, j, r)); }
    else { h->err = "rdm2: |dx|+|dy| must be 1"; return CTM_ERR_ARG; }
    rho.resize(r.size());
    if (!swap) rho = r;
    else
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b)
                for (int c = 0; c < d; ++c)
                    for (int e = 0; e < d; ++e)
                        rho[((size_t)(a * d + b)) * d * d + (c * d + e)] = r[((size_t)(b * d + a)) * d * d + (e * d + c)];
    normalise_trace(rho, d * d);
    return CTM_OK;
}

// sum_i x[i] y[i] (device arrays) to the host
ctm_status dot_host(ctm_ctx* h, const double* x, const double* y, size_t n, double* out) {
    CK(ctm::dot(x, y, n, h->scal, h->dotws, h->stream));
    CK(cudaMemcpyAsync(out, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return CTM_OK;
}

// Closed strip of a 2x2 block with no sites: the corners cTL, cTR, cBR, cBL
// around it and, between them, two pairs of edges facing each other across
// the block, each edge's ket/bra legs joined to those of the edge opposite.
// With (cTL, e1, e2, cTR) = (C1, T1(TL), T1(TR), C2) on top and
// (cBR, e3, e4, cBL) = (C3, T3(BR), T3(BL), C4) below this is Z_20; with the
// right and left columns fed in the same roles it is Z_02.
//   top[a,(u,U),(v,V),f] = cTL[a,b] e1[b,(u,U),c] e2[c,(v,V),e] cTR[e,f]
//   bot[f,(v,V),(u,U),a] = cBR[f,g] e3[g,(v,V),h] e4[h,(u,U),k] cBL[k,a]
//   Z = sum top[a,u,U,v,V,f] bot[f,v,V,u,U,a]
ctm_status strip_value(ctm_ctx* h, const double* cTL, const double* e1, const double* e2, const double* cTR,
                       const double* cBR, const double* e3, const double* e4, const double* cBL, double* z) {
    const int chi = h->chi, N = h->N, D = h->D;
    const int ND2 = N * D * D;
    CKS(gemm(h, false, false, chi, N, chi, cTL, chi, e1, N, h->X1, N));
    CKS(gemm(h, false, false, N, N, chi, h->X1, chi, e2, N, h->E[0], N));
    CKS(gemm(h, false, false, ND2, chi, chi, h->E[0], chi, cTR, chi, h->E[1], chi));
    CKS(gemm(h, false, false, chi, N, chi, cBR, chi, e3, N, h->X1, N));
    CKS(gemm(h, false, false, N, N, chi, h->X1, chi, e4, N, h->E[0], N));
    CKS(gemm(h, false, false, ND2, chi, chi, h->E[0], chi, cBL, chi, h->E[2], chi));
    CKS(perm(h, h->E[2], h->E[0], {chi, D, D, D, D, chi}, {5, 3, 4, 1, 2, 0}));
    return dot_host(h, h->E[1], h->E[0], (size_t)N * N, z);
}

// ln kappa per site (Sec. 2.2 norm network): for the 2x2 block TL = 2,
// TR = 3, BL = 0, BR = 1, kappa_block = Z_22 Z_00 / (Z_20 Z_02) where Z_22 is
// the block with its full environment (= Tr(H_u^T H_d) of the cut through
// it), Z_00 the four corners joined directly, Z_20 / Z_02 the row / column
// strips without sites; ln kappa per site = ln(kappa_block) / 4.  Every
// environment normalisation cancels in the ratio.
ctm_status log_norm_per_site(ctm_ctx* h, double* out) {
    const int chi = h->chi, N = h->N;
    const int TL = 2, TR = 3, BR = 1, BL = 0;
    double z00 = 0, z20 = 0, z02 = 0, z22 = 0;
    // Z_00 = Tr(C1 C2 C3 C4) = sum P[a,b] Q[b,a], P = C1 C2, Q = C3 C4
    CKS(gemm(h, false, false, chi, chi, chi, h->env[TL][C1], chi, h->env[TR][C2], chi, h->newC1, chi));
    CKS(gemm(h, false, false, chi, chi, chi, h->env[BR][C3], chi, h->env[BL][C4], chi, h->newC4, chi));
    CKS(perm(h, h->newC4, h->corners, {chi, chi}, {1, 0}));
    CKS(dot_host(h, h->newC1, h->corners, (size_t)chi * chi, &z00));
    CKS(strip_value(h, h->env[TL][C1], h->env[TL][T1], h->env[TR][T1], h->env[TR][C2], h->env[BR][C3],
                    h->env[BR][T3], h->env[BL][T3], h->env[BL][C4], &z20));
    // columns: right (C2, T2(TR), T2(BR), C3) and left (C4, T4(BL), T4(TL), C1)
    CKS(strip_value(h, h->env[TR][C2], h->env[TR][T2], h->env[BR][T2], h->env[BR][C3], h->env[BL][C4],
                    h->env[BL][T4], h->env[TL][T4], h->env[TL][C1], &z02));
    // Z_22 = Tr(H_u^T H_d) over the cut between rows 0 and 1 at column 0.
    // The four corners of a cut are held as H_u = E_ul E_ur and
    // H_d^T = E_br E_bl (the lower two corners transposed), so
    // Z_22 = Tr(E_ul E_ur E_br E_bl) = sum_ab (E_ul E_ur)[a,b] (E_br E_bl)[b,a].
    CKS(enlarged_corner(h, TL, 0, h->E[0]));
    CKS(enlarged_corner(h, TR, 1, h->E[1]));
    CKS(enlarged_corner(h, BR, 2, h->E[2]));
    CKS(enlarged_corner(h, BL, 3, h->E[3]));
    CKS(gemm(h, false, false, N, N, N, h->E[0], N, h->E[1], N, h->S1, N));
    CKS(gemm(h, false, false, N, N, N, h->E[2], N, h->E[3], N, h->S3, N));
    CKS(perm(h, h->S3, h->S2, {N, N}, {1, 0}));
    CKS(dot_host(h, h->S1, h->S2, (size_t)N * N, &z22));
    const double ratio = z22 * z00 / (z20 * z02);
    if (!(ratio > 0.0) || !std::isfinite(ratio)) {
        char buf[200];
        snprintf(buf, sizeof(buf), "ln kappa: Z22 Z00 / (Z20 Z02) = %.3e is not a positive finite number", ratio);
        h->err = buf;
        return CTM_ERR_NONFINITE;
    }
    *out = 0.25 * std::log(ratio);
    return CTM_OK;
}

// ----------------------------------------------------------------------------
// correlation functions and the transfer-matrix spectrum (Sec. 5.3)
//
// Strips run along +x' of a frame: frame 0 along +x, frame 3 (the lattice
// rotated clockwise, where the original bottom edge is the frame's left
// edge) along +y.  In frame m the roles C1..T4 are played by env[Cw(m)],
// env[Tw(m)], ..., env[Tw(m+3)] and the site tensor by A[i][m].  A strip
// vector L[b, l, l', t] (chi x D x D x chi) holds the contracted part left of
// a column: b the open chi index toward the next T3, (l, l') the ket and bra
// legs toward the next site, t the open chi index toward the next T1.
//   left edge      L0 = C4 T4 C1
//   one column     L'[b', r, r', t'] = L[b, l, l', t] T1[t, u, u', t']
//                     Aket[s, l, u, r, d] Abra[s, l', u', r', d'] T3[b', d, d', b]
//   right edge     R[t, r, r', b] = C2 T2 C3, closed as sum L[b,r,r',t] R[t,r,r',b]
// The column is corner_core with (T1, L) in the roles of (C1 T1, T4) --
// E[(b,d,d'), (t',r,r')] -- followed by one product with T3.
// ----------------------------------------------------------------------------
void frame_pos(int m, int i, int* x, int* y) {
    for (int p = 0; p < 4; ++p)
        if (FM.site(m, p % 2, p / 2) == i) {
            *x = p % 2;
            *y = p / 2;
            return;
        }
    *x = *y = 0;
}

struct CorrBufs {
    double* v[9];      // strip vectors
    double* ket[4];    // Alu layouts [l,u,t,r,d] with an operator on the ket
    double* op[3];     // d x d operators
};
ctm_status corr_bufs(ctm_ctx* h, CorrBufs* b) {
    const size_t T = (size_t)h->chi * h->N, A = (size_t)h->d * h->D * h->D * h->D * h->D;
    const size_t dd = (size_t)h->d * h->d;
    if (!h->cv) CKS(allocd(h, &h->cv, 9 * T + 4 * A + 3 * dd));
    for (int j = 0; j < 9; ++j) b->v[j] = h->cv + j * T;
    for (int j = 0; j < 4; ++j) b->ket[j] = h->cv + 9 * T + j * A;
    for (int j = 0; j < 3; ++j) b->op[j] = h->cv + 9 * T + 4 * A + j * dd;
    return CTM_OK;
}

// L0[b, l, l', t] = C4[b, n] T4[n, l, l', a] C1[a, t] of site i in frame m
ctm_status strip_left(ctm_ctx* h, int m, int i, double* out, double* tmp) {
    const int chi = h->chi, N = h->N;
    double** e = h->env[i];
    CKS(gemm(h, false, false, chi, N, chi, e[Cw(m + 3)], chi, e[Tw(m + 3)], N, tmp, N));
    return gemm(h, false, false, N, chi, chi, tmp, chi, e[Cw(m)], chi, out, chi);
}
// R[t, r, r', b] = C2[t, e] T2[e, r, r', f] C3[f, b], stored as [b, r, r', t]
ctm_status strip_right(ctm_ctx* h, int m, int i, double* out, double* tmp, double* tmp2) {
    const int chi = h->chi, N = h->N, D = h->D;
    double** e = h->env[i];
    CKS(gemm(h, false, false, chi, N, chi, e[Cw(m + 1)], chi, e[Tw(m + 1)], N, tmp, N));
    CKS(gemm(h, false, false, N, chi, chi, tmp, chi, e[Cw(m + 2)], chi, tmp2, chi));
    return perm(h, tmp2, out, {chi, D, D, chi}, {3, 1, 2, 0});
}
// one column of site i in frame m: out = L (T1 Aket Abra T3); ket in Alu layout
ctm_status strip_column(ctm_ctx* h, int m, int i, const double* L, const double* ket, double* out, double* t3p,
                        double* tmp) {
    const int chi = h->chi, N = h->N, D = h->D;
    double** e = h->env[i];
    CKS(corner_core(h, e[Tw(m)], L, h->A[i][m & 3], ket, h->E[0], false));
    // T3[k, d, d', b] -> [k, b, d, d'];  out'[k, (t', r, r')] = T3p[k, (b,d,d')] E[(b,d,d'), (t',r,r')]
    CKS(perm(h, e[Tw(m + 2)], t3p, {chi, D, D, chi}, {0, 3, 1, 2}));
    CKS(gemm(h, false, false, chi, N, N, t3p, N, h->E[0], N, tmp, N));
    return perm(h, tmp, out, {chi, chi, D, D}, {0, 2, 3, 1});
}
// ket of site i in frame m with O[t, s] applied, in the Alu layout [l,u,t,r,d]
// (tmp: d D^4 doubles)
ctm_status ket_with_op(ctm_ctx* h, int m, int i, const double* op, double* out, double* tmp) {
    const int d = h->d, D = h->D, D4 = D * D * D * D;
    CK(ctm::dgemm(false, false, d, D4, d, 1.0, op, d, h->A[i][m & 3], D4, 0.0, tmp, D4, h->stream, nullptr, 0));
    return perm(h, tmp, out, {d, D, D, D, D}, {1, 2, 0, 3, 4});
}
// L /= max|L| and X /= max|L| (the same factor: the ratio of two strips is kept)
ctm_status rescale_pair(ctm_ctx* h, double* L, double* X) {
    const size_t n = (size_t)h->chi * h->N;
    CK(cudaMemsetAsync(h->maxbits + 8, 0, sizeof(unsigned long long), h->stream));
    CK(ctm::maxabs(L, n, h->maxbits + 8, h->stream));
    CK(ctm::scale_by_max(X, n, h->maxbits + 8, h->flag, h->stream));
    CK(ctm::scale_by_max(L, n, h->maxbits + 8, h->flag, h->stream));
    return CTM_OK;
}

// C[dir][site][r]: numerators and denominators on the device, one copy back
ctm_status correlation(ctm_ctx* h, const double* opA_h, const double* opB_h, int rmax, double* out) {
    CKS(check_ready(h));
    CorrBufs b;
    CKS(corr_bufs(h, &b));
    const int d = h->d;
    const size_t n = (size_t)h->chi * h->N, nvals = (size_t)2 * 4 * (rmax + 1);
    double* nd = nullptr;  // [dir][site][r][num, den]
    CKS(allocd_tmp(h, &nd, 2 * nvals));
    ctm_status st = CTM_OK;
    auto body = [&]() -> ctm_status {
        CK(cudaMemcpyAsync(b.op[0], opA_h, sizeof(double) * d * d, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(b.op[1], opB_h, sizeof(double) * d * d, cudaMemcpyHostToDevice, h->stream));
        // A B (B acts first)
        CK(ctm::dgemm(false, false, d, d, d, 1.0, b.op[0], d, b.op[1], d, 0.0, b.op[2], d, h->stream, nullptr, 0));
        double *LA = b.v[0], *L1 = b.v[1], *XB = b.v[2], *X1 = b.v[3], *tmp = b.v[4], *tmp2 = b.v[5];
        double *t3p = b.v[6], *R = b.v[7], *L0 = b.v[8];
        for (int dir = 0; dir < 2; ++dir) {
            const int m = dir == 0 ? 0 : 3;
            for (int i0 = 0; i0 < 4; ++i0) {
                int x0, y0;
                frame_pos(m, i0, &x0, &y0);
                double* res = nd + 2 * ((size_t)(dir * 4 + i0) * (rmax + 1));
                // r = 0: <A B> at r0
                CKS(strip_left(h, m, i0, L0, tmp));
                CKS(strip_right(h, m, i0, R, tmp, tmp2));
                CKS(ket_with_op(h, m, i0, b.op[2], b.ket[0], b.ket[3]));
                CKS(strip_column(h, m, i0, L0, b.ket[0], XB, t3p, tmp));
                CKS(strip_column(h, m, i0, L0, h->Alu[i0][m & 3], L1, t3p, tmp));
                CK(ctm::dot(XB, R, n, res + 0, h->dotws, h->stream));
                CK(ctm::dot(L1, R, n, res + 1, h->dotws, h->stream));
                if (rmax == 0) continue;
                CKS(ket_with_op(h, m, i0, b.op[0], b.ket[0], b.ket[3]));
                CKS(strip_column(h, m, i0, L0, b.ket[0], LA, t3p, tmp));
                CKS(rescale_pair(h, L1, LA));
                for (int r = 1; r <= rmax; ++r) {
                    const int s = FM.site(m, x0 + r, y0);
                    CKS(strip_right(h, m, s, R, tmp, tmp2));
                    CKS(ket_with_op(h, m, s, b.op[1], b.ket[1], b.ket[3]));
                    CKS(strip_column(h, m, s, LA, b.ket[1], XB, t3p, tmp));
                    CKS(strip_column(h, m, s, L1, h->Alu[s][m & 3], X1, t3p, tmp));
                    CK(ctm::dot(XB, R, n, res + 2 * r, h->dotws, h->stream));
                    CK(ctm::dot(X1, R, n, res + 2 * r + 1, h->dotws, h->stream));
                    if (r == rmax) break;
                    CKS(strip_column(h, m, s, LA, h->Alu[s][m & 3], XB, t3p, tmp));
                    std::swap(LA, XB);
                    std::swap(L1, X1);
                    CKS(rescale_pair(h, L1, LA));
                }
            }
        }
        std::vector<double> hv(2 * nvals);
        CK(cudaMemcpyAsync(hv.data(), nd, sizeof(double) * 2 * nvals, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        CKS(read_flag(h));
        for (size_t j = 0; j < nvals; ++j) out[j] = hv[2 * j] / hv[2 * j + 1];
        return CTM_OK;
    };
    st = body();
    cudaStreamSynchronize(h->stream);
    cudaFree(nd);
    return st;
}

// Leading eigenvalues of the period transfer matrix of row `index` of frame
// m: explicitly restarted block Arnoldi.  A cycle builds an orthonormal
// basis Q of the block Krylov space {V, T V, ..., T^(p-1) V} (blocks of
// `blk` vectors as rows, m = blk p <= 32) by block Gram-Schmidt (two passes,
// and the new block orthogonalised once more after its QR, so that a
// breakdown -- a residual at rounding level -- still yields an orthonormal
// block), with H = Q^T T Q assembled from the projection coefficients; the
// eigenvalues of H (Rayleigh-Ritz) are the estimates, and the next cycle
// restarts from the real parts of the leading Ritz vectors.  (Subspace
// iteration, tried first, needed ~4x the products on clustered spectra.)
ctm_status transfer_spectrum(ctm_ctx* h, int dir, int index, int nev, int blk, int max_iter, double tol,
                             double* out, int* iters, double* change) {
    CKS(check_ready(h));
    CorrBufs b;
    CKS(corr_bufs(h, &b));
    const int m = dir == 0 ? 0 : 3;
    int xs, ys;
    frame_pos(m, dir == 0 ? index * 2 : index, &xs, &ys);  // site (0, index) or (index, 0)
    const int s0 = FM.site(m, 0, ys), s1 = FM.site(m, 1, ys);
    const size_t n = (size_t)h->chi * h->N;
    const int p = std::min(ctm::small_eig_max() / blk, (int)(n / blk));  // Krylov blocks per cycle
    const int mk = blk * p;                                              // basis size
    if (p < 2) {
        h->err = "transfer spectrum: block too large for a Krylov space of two blocks";
        return CTM_ERR_ARG;
    }
    double *Qa = nullptr, *W = nullptr, *Y = nullptr, *Qn = nullptr, *Rr = nullptr, *Cc = nullptr, *H = nullptr;
    double *ev = nullptr, *evr = nullptr, *Yr = nullptr;
    void* qws = nullptr;
    int* est = nullptr;
    ctm_status st = CTM_OK;
    auto body = [&]() -> ctm_status {
        CKS(allocd_tmp(h, &Qa, (size_t)mk * n));
        CKS(allocd_tmp(h, &W, (size_t)blk * n));
        CKS(allocd_tmp(h, &Y, (size_t)blk * n));
        CKS(allocd_tmp(h, &Qn, (size_t)blk * n));
        CKS(allocd_tmp(h, &Rr, (size_t)blk * blk));
        CKS(allocd_tmp(h, &Cc, (size_t)mk * blk));
        CKS(allocd_tmp(h, &H, (size_t)mk * mk));
        CKS(allocd_tmp(h, &ev, (size_t)4 * mk + 8));
        CKS(allocd_tmp(h, &evr, (size_t)2 * mk));
        CKS(allocd_tmp(h, &Yr, (size_t)blk * mk));
        if (cudaMalloc(&qws, ctm::qr_ws_bytes((int)n, blk)) != cudaSuccess) {
            cudaGetLastError();
            h->err = "transfer spectrum: out of device memory";
            return CTM_ERR_OOM;
        }
        est = (int*)(ev + 4 * mk);
        double *tmp = b.v[4], *t3p = b.v[6], *mid = b.v[7];
        const int nn = (int)n;
        // rows of dst (blk x n) = an orthonormal basis of the rows of src
        auto orth = [&](const double* src, double* dst) -> ctm_status {
            CKS(perm(h, src, Y, {blk, nn}, {1, 0}));
            CK(ctm::qr(Y, nn, blk, Qn, Rr, qws, h->stream, h->flag + 1));
            return perm(h, Qn, dst, {nn, blk}, {1, 0});
        };
        // W -= (Qa[0:L] W^T)^T Qa[0:L], the coefficients into Cc (L x blk); twice
        auto project = [&](int L, double* Hcol) -> ctm_status {
            for (int pass = 0; pass < 2; ++pass) {
                CK(ctm::dgemm(false, true, L, blk, nn, 1.0, Qa, nn, W, nn, 0.0, Cc, blk, h->stream, h->splitk,
                              h->splitk_n));
                CK(ctm::dgemm(true, false, blk, nn, L, -1.0, Cc, blk, Qa, nn, 1.0, W, nn, h->stream, nullptr, 0));
                if (Hcol) CK(ctm::add_block(Cc, L, blk, blk, Hcol, mk, h->stream));
            }
            return CTM_OK;
        };
        CK(ctm::rng_normal(W, (size_t)blk * n, h->opt.seed, 0x5452414eull + h->rng_counter++, h->stream));
        CKS(orth(W, Qa));
        std::vector<double> prev(nev, -1.0), cur(4 * mk);
        double delta = INFINITY;
        int it = 0;
        st = CTM_NOT_CONVERGED;
        for (it = 1; it <= max_iter; ++it) {
            CK(cudaMemsetAsync(H, 0, sizeof(double) * mk * mk, h->stream));
            for (int sb = 0; sb < p; ++sb) {
                for (int j = 0; j < blk; ++j) {
                    const double* v = Qa + ((size_t)sb * blk + j) * n;
                    CKS(strip_column(h, m, s0, v, h->Alu[s0][m & 3], mid, t3p, tmp));
                    CKS(strip_column(h, m, s1, mid, h->Alu[s1][m & 3], W + (size_t)j * n, t3p, tmp));
                }
                const int L = (sb + 1) * blk;
                CKS(project(L, H + (size_t)sb * blk));
                if (sb + 1 < p) {
                    // W = Q_new R: R is the subdiagonal block of H
                    CKS(perm(h, W, Y, {blk, nn}, {1, 0}));
                    CK(ctm::qr(Y, nn, blk, Qn, Rr, qws, h->stream, h->flag + 1));
                    CK(ctm::add_block(Rr, blk, blk, blk, H + (size_t)L * mk + (size_t)sb * blk, mk, h->stream));
                    CKS(perm(h, Qn, W, {nn, blk}, {1, 0}));
                    CKS(project(L, nullptr));       // the new block once more against the basis
                    CKS(orth(W, Qa + (size_t)L * n));
                }
            }
            CK(ctm::small_eig(H, mk, mk, 2.0, ev, est, h->stream, evr));
            CK(cudaMemcpyAsync(cur.data(), ev, sizeof(double) * 4 * mk, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            // change of the moduli |lambda_i / lambda_0| (what e_i and xi are
            // made of): among eigenvalues of equal modulus -- a complex pair,
            // or +-lambda -- the order, and so the complex ratio, may swap
            // from one cycle to the next
            delta = 0.0;
            for (int i = 0; i < nev; ++i) {
                const double mod = std::hypot(cur[i], cur[mk + i]);
                delta = std::max(delta, std::fabs(mod - prev[i]));
                prev[i] = mod;
            }
            if (!(delta == delta)) delta = INFINITY;
            if (delta < tol) {
                st = CTM_OK;
                break;
            }
            // restart: V = orth(Y_ritz Q), Y_ritz the real basis of the leading Ritz vectors
            CK(ctm::ritz_basis(H, mk, mk, evr, blk, Yr, h->stream));
            CK(ctm::dgemm(false, false, blk, nn, mk, 1.0, Yr, mk, Qa, nn, 0.0, W, nn, h->stream, nullptr, 0));
            CKS(orth(W, Qa));
        }
        CKS(read_flag(h));
        if (iters) *iters = std::min(it, max_iter);
        if (change) *change = delta;
        for (int i = 0; i < nev; ++i) {
            out[i] = cur[i];
            out[nev + i] = cur[mk + i];
            out[2 * nev + i] = cur[2 * mk + i];
            out[3 * nev + i] = cur[3 * mk + i];
        }
        return st;
    };
    st = body();
    cudaStreamSynchronize(h->stream);
    for (double* q : {Qa, W, Y, Qn, Rr, Cc, H, ev, evr, Yr}) cudaFree(q);
    cudaFree(qws);
    return st;
}

thread_local std::string g_err;

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* ctm_status_string(ctm_status s) {
    switch (s) {
        case CTM_OK: return "ok";
        case CTM_NOT_CONVERGED: return "not converged";
        case CTM_ERR_ARG: return "invalid argument";
        case CTM_ERR_OOM: return "out of device memory";
        case CTM_ERR_CUDA: return "CUDA error";
        case CTM_ERR_NONFINITE: return "non-finite values";
        case CTM_ERR_TIMEOUT: return "device wait timed out";
        case CTM_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

const char* ctm_last_error(ctm_handle h) { return h ? h->err.c_str() : g_err.c_str(); }

ctm_status ctm_default_options(ctm_options* o) {
    if (!o) return CTM_ERR_ARG;
    o->chi = 16;
    o->max_sweeps = 100;
    o->tol = 1e-10;
    o->precision = CTM_FP64;
    o->ozaki_slices = 5;
    o->rsvd_oversample = 0;
    o->rsvd_power_iters = 2;
    o->sv_cutoff_rel = 1e-12;
    o->seed = 0;
    o->exact_svd_max_n = 256;
    o->rsvd_warm_start = 1;
    o->conv_measure = 0;
    o->fp64_refine = 0;
    o->batch_cuts = 1;
    return CTM_OK;
}

static ctm_status validate(int d, int D, const ctm_options* o) {
    if (!o || d < 1 || D < 1 || o->chi < 1 || d > 64 || D > 64) return CTM_ERR_ARG;
    if (o->precision != CTM_FP64 && tc_mode_of(o->precision) < 0) return CTM_ERR_ARG;
    if (o->rsvd_power_iters < 0) return CTM_ERR_ARG;
    if (o->conv_measure != 0 && o->conv_measure != 1) return CTM_ERR_ARG;
    if (o->precision == CTM_OZAKI_BF16 && (o->ozaki_slices < 2 || o->ozaki_slices > 6)) return CTM_ERR_ARG;
    const long long N = (long long)o->chi * D * D;
    if ((long long)d * d * N * N >= (1ll << 32)) return CTM_ERR_ARG;  // index range of the kernels
    return CTM_OK;
}

ctm_status ctm_footprint_bytes(int d, int D, const ctm_options* o, size_t* bytes) {
    if (!bytes || validate(d, D, o) != CTM_OK) return CTM_ERR_ARG;
    *bytes = footprint(d, D, *o);
    return CTM_OK;
}

namespace {
ctm_status create(int Lx, int Ly, int d, int D, const ctm_options* o, void* stream, void* arena, size_t arena_n,
                  ctm_handle* out);
}

ctm_status ctm_create(int Lx, int Ly, int d, int D, const ctm_options* o, void* stream, ctm_handle* out) {
    return create(Lx, Ly, d, D, o, stream, nullptr, 0, out);
}

ctm_status ctm_create_in(int Lx, int Ly, int d, int D, const ctm_options* o, void* stream, void* arena,
                         size_t arena_bytes, ctm_handle* out) {
    if (!arena || ((uintptr_t)arena & 255) != 0) {
        g_err = "ctm_create_in: the arena must be a device pointer aligned to 256 bytes";
        return CTM_ERR_ARG;
    }
    if (o && validate(d, D, o) == CTM_OK && arena_bytes < footprint(d, D, *o)) {
        g_err = "ctm_create_in: the arena is smaller than ctm_footprint_bytes";
        return CTM_ERR_ARG;
    }
    return create(Lx, Ly, d, D, o, stream, arena, arena_bytes, out);
}

namespace {
ctm_status create(int Lx, int Ly, int d, int D, const ctm_options* o, void* stream, void* arena, size_t arena_n,
                  ctm_handle* out) {
    if (!out) return CTM_ERR_ARG;
    *out = nullptr;
    if (Lx != 2 || Ly != 2) {
        g_err = "ctm_create: only the 2x2 unit cell (Lx = Ly = 2) is built";
        return CTM_ERR_ARG;
    }
    if (o && o->precision == CTM_OZAKI_INT8) {
        g_err = "ctm_create: CTM_OZAKI_INT8 is not built (INT8 tensor-core slices)";
        return CTM_ERR_ARG;
    }
    if (validate(d, D, o) != CTM_OK) {
        g_err = "ctm_create: invalid dimensions or options";
        return CTM_ERR_ARG;
    }
    ctm_ctx* h = new (std::nothrow) ctm_ctx();
    if (!h) return CTM_ERR_OOM;
    h->arena = (char*)arena;
    h->arena_n = arena_n;
    h->d = d;
    h->D = D;
    h->opt = *o;
    h->chi = o->chi;
    h->N = o->chi * D * D;
    h->k = rsvd_k(h->N, h->chi, *o);
    h->q = o->rsvd_power_iters;
    if (stream) h->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            g_err = "cudaStreamCreate failed";
            delete h;
            return CTM_ERR_CUDA;
        }
        h->own_stream = true;
    }
    Sizes z = sizes_of(d, D, h->chi, h->k);
    const size_t N = h->N;
    ctm_status st = CTM_OK;
    auto A_ = [&](double** p, size_t n) { if (st == CTM_OK) st = allocd(h, p, n); };
    for (int i = 0; i < 4; ++i)
        for (int r = 0; r < 4; ++r) { A_(&h->A[i][r], z.A); A_(&h->Alu[i][r], z.A); }
    for (int i = 0; i < 4; ++i)
        for (int w = 0; w < 8; ++w) A_(&h->env[i][w], (w & 1) ? z.T : z.C);
    A_(&h->X1, z.T);
    A_(&h->S1, z.open);
    A_(&h->S3, z.open);
    A_(&h->S2, (size_t)d * z.NN);
    for (int c = 0; c < (o->batch_cuts ? 8 : 4); ++c) A_(&h->E[c], z.NN);
    if (o->batch_cuts) {
        A_(&h->Qm1, z.Nk); A_(&h->Qb1, z.Nk); A_(&h->G1, z.kk); A_(&h->Us1, z.kk); A_(&h->Ws1, z.kk);
        A_(&h->Sv1, h->k);
        if (st == CTM_OK) st = alloc(h, &h->svd2_ws, svd2_ws_bytes(h->k));
    }
    for (int s = 0; s < 2; ++s) { A_(&h->Pup[s], z.Nchi); A_(&h->PdnT[s], z.Nchi); }
    A_(&h->Om, z.Nk); A_(&h->Yb, z.Nk); A_(&h->Zb, z.Nk); A_(&h->Qm, z.Nk); A_(&h->Qm2, z.Nk); A_(&h->Qb, z.Nk);
    A_(&h->Rb, z.kk); A_(&h->G, z.kk); A_(&h->Us, z.kk); A_(&h->Ws, z.kk);
    A_(&h->Sv, h->k); A_(&h->inv, h->k);
    const size_t tk = std::max(z.Nk, z.Nchi);
    A_(&h->Uc, z.Nchi); A_(&h->Vc, z.Nk); A_(&h->t1, tk); A_(&h->t2, tk);
    A_(&h->newC1, z.C); A_(&h->newC4, z.C); A_(&h->newT4, z.T); A_(&h->tmpT, z.T);
    A_(&h->Lh, z.Nchi * d * d); A_(&h->Rh, z.Nchi * d * d);
    A_(&h->rho, std::max<size_t>(64 * 64, (size_t)d * d * d * d));
    h->splitk_n = (size_t)1 << 24;
    A_(&h->splitk, h->splitk_n);
    A_(&h->spec, 16 * (size_t)h->chi);
    A_(&h->corners, 16 * z.C);
    if (st == CTM_OK) st = alloc(h, &h->qr_ws, qr_ws_bytes(h->N, h->k));
    if (st == CTM_OK) st = alloc(h, &h->svd_ws, svd_ws_bytes(h->k));
    if (st == CTM_OK) st = alloc(h, &h->sval_ws, svals_ws_bytes(h->chi, 16));
    if (st == CTM_OK) st = alloc(h, (void**)&h->maxbits, 64 * sizeof(unsigned long long));
    if (st == CTM_OK) st = alloc(h, (void**)&h->flag, 64);
    if (st == CTM_OK) st = allocd(h, &h->dotws, ctm::dot_ws_doubles());
    if (st == CTM_OK) st = allocd(h, &h->scal, 8);
    if (o->rsvd_warm_start && h->k < h->N)
        for (int c = 0; c < 16 && st == CTM_OK; ++c) st = allocd(h, &h->warmV[c], z.Nk);
    const int tmode = tc_mode_of(o->precision), tsl = tc_slices_of(*o);
    if (tmode >= 0) h->tc_prec = o->precision;
    if (st == CTM_OK && tmode >= 0) {
        const OzBounds zb = oz_bounds(d, D, h->chi, h->k, tsl, tmode);
        h->ozA_n = zb.a;
        h->ozB_n = zb.b;
        h->ozW_n = std::max<size_t>(zb.w, 256);
        st = alloc(h, &h->ozA, h->ozA_n);
        if (st == CTM_OK) st = alloc(h, &h->ozB, h->ozB_n);
        if (st == CTM_OK) st = alloc(h, &h->ozW, h->ozW_n);
        for (int c = 0; c < (o->batch_cuts ? 16 : 8) && st == CTM_OK; ++c) {
            h->ozc[c].ptr = h->E[c / 2];
            h->ozc[c].trans = (c & 1) != 0;
            st = alloc(h, &h->ozc[c].buf, tc_split_bytes(h->N, h->N, tmode, tsl));
        }
    }
    if (st != CTM_OK) {
        g_err = h->err;
        ctm_destroy(h);
        return st;
    }
    if (cudaMemsetAsync(h->flag, 0, 64, h->stream) != cudaSuccess) {
        g_err = "cudaMemset failed";
        ctm_destroy(h);
        return CTM_ERR_CUDA;
    }
    *out = h;
    return CTM_OK;
}
}  // namespace

ctm_status ctm_destroy(ctm_handle h) {
    if (!h) return CTM_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (void* p : h->allocs) cudaFree(p);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return CTM_OK;
}

ctm_status ctm_set_tensor(ctm_handle h, int site, const double* A, int on_device) {
    if (!h || !A || site < 0 || site > 3) return CTM_ERR_ARG;
    const int d = h->d, D = h->D;
    const size_t n = (size_t)d * D * D * D * D;
    CK(cudaMemcpyAsync(h->A[site][0], A, n * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    for (int r = 1; r < 4; ++r) CKS(perm(h, h->A[site][r - 1], h->A[site][r], {d, D, D, D, D}, {0, 2, 3, 4, 1}));
    for (int r = 0; r < 4; ++r) CKS(perm(h, h->A[site][r], h->Alu[site][r], {d, D, D, D, D}, {1, 2, 0, 3, 4}));
    CK(cudaStreamSynchronize(h->stream));
    h->have_A[site] = true;
    for (bool& w : h->warm_valid) w = false;
    return CTM_OK;
}

ctm_status ctm_set_env(ctm_handle h, int site, int which, const double* t, int on_device) {
    if (!h || !t || site < 0 || site > 3 || which < 0 || which > 7) return CTM_ERR_ARG;
    const size_t n = (which & 1) ? (size_t)h->chi * h->D * h->D * h->chi : (size_t)h->chi * h->chi;
    CK(cudaMemcpyAsync(h->env[site][which], t, n * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->env_set |= 1u << (site * 8 + which);
    for (bool& w : h->warm_valid) w = false;
    return CTM_OK;
}

ctm_status ctm_get_env(ctm_handle h, int site, int which, double* t, int on_device) {
    if (!h || !t || site < 0 || site > 3 || which < 0 || which > 7) return CTM_ERR_ARG;
    const size_t n = (which & 1) ? (size_t)h->chi * h->D * h->D * h->chi : (size_t)h->chi * h->chi;
    CK(cudaMemcpyAsync(t, h->env[site][which], n * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return CTM_OK;
}

ctm_status ctm_sweep(ctm_handle h, int n) {
    if (!h || n < 0) return CTM_ERR_ARG;
    CKS(check_ready(h));
    const long long capped0 = h->jacobi_capped;
    for (int s = 0; s < n; ++s) CKS(one_sweep(h));
    const ctm_status st = read_flag(h);
    prof_collect(h);
    if (st == CTM_OK && h->jacobi_capped > capped0) {
        h->err = "a projector SVD reached the Jacobi sweep cap (results usable, rotations not fully converged)";
        return CTM_NOT_CONVERGED;
    }
    return st;
}

ctm_status ctm_sweep_async(ctm_handle h, int n) {
    if (!h || n < 0) return CTM_ERR_ARG;
    CKS(check_ready(h));
    for (int s = 0; s < n; ++s) CKS(one_sweep(h));
    return CTM_OK;
}

ctm_status ctm_sync(ctm_handle h) {
    if (!h) return CTM_ERR_ARG;
    const ctm_status st = read_flag(h);
    prof_collect(h);
    return st;
}

ctm_status ctm_batch_sweep(const ctm_handle* hs, int n, int sweeps) {
    if (!hs || n < 0 || sweeps < 0) return CTM_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return CTM_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return CTM_ERR_ARG;
        CKS(check_ready(hs[i]));
    }
    ctm_status first = CTM_OK;
    for (int s = 0; s < sweeps && first == CTM_OK; ++s)
        for (int i = 0; i < n; ++i) {
            const ctm_status st = one_sweep(hs[i]);
            if (st != CTM_OK && first == CTM_OK) first = st;
        }
    for (int i = 0; i < n; ++i) {
        const ctm_status st = read_flag(hs[i]);
        prof_collect(hs[i]);
        if (st != CTM_OK && first == CTM_OK) first = st;
    }
    return first;
}

ctm_status ctm_spectrum_delta(ctm_handle h, double* delta) {
    if (!h || !delta) return CTM_ERR_ARG;
    CKS(check_ready(h));
    CKS(read_flag(h));
    std::vector<double> cur;
    CKS(spectra(h, cur));
    double d = INFINITY;
    if (h->last_spec.size() == cur.size()) {
        d = 0.0;
        for (size_t i = 0; i < cur.size(); ++i) d = std::max(d, std::fabs(cur[i] - h->last_spec[i]));
    }
    h->last_spec.swap(cur);
    *delta = d;
    return CTM_OK;
}

ctm_status ctm_run(ctm_handle h, int* sweeps_done, double* last_delta) {
    if (!h) return CTM_ERR_ARG;
    CKS(check_ready(h));
    std::vector<double> prev, cur;
    const bool loops = h->opt.conv_measure == 1;
    auto measure = [&](std::vector<double>& v) { return loops ? loop_moments(h, v) : spectra(h, v); };
    CKS(measure(prev));
    double delta = INFINITY;
    int n = 0;
    ctm_status st = CTM_NOT_CONVERGED;
    for (n = 1; n <= h->opt.max_sweeps; ++n) {
        CKS(one_sweep(h));
        CKS(read_flag(h));
        CKS(measure(cur));
        delta = 0.0;
        for (size_t i = 0; i < cur.size(); ++i) {
            const double x = std::fabs(cur[i] - prev[i]);
            delta = (x != x) ? INFINITY : std::max(delta, x);
        }
        prev.swap(cur);
        if (delta < h->opt.tol) { st = CTM_OK; break; }
        if (h->opt.fp64_refine && tc_mode_of(h->opt.precision) >= 0 && delta < refine_at(h->opt)) {
            // the tensor-core products' rounding keeps the measure from
            // falling much below this: the remaining sweeps run in FP64
            CKS(set_precision(h, CTM_FP64));
        }
    }
    if (n > h->opt.max_sweeps) n = h->opt.max_sweeps;
    if (sweeps_done) *sweeps_done = n;
    if (last_delta) *last_delta = delta;
    return st;
}

ctm_status ctm_set_precision(ctm_handle h, int precision) {
    if (!h || (precision != CTM_FP64 && tc_mode_of(precision) < 0)) return CTM_ERR_ARG;
    return set_precision(h, precision);
}

ctm_status ctm_loop_delta(ctm_handle h, double* delta) {
    if (!h || !delta) return CTM_ERR_ARG;
    CKS(check_ready(h));
    CKS(read_flag(h));
    std::vector<double> cur;
    CKS(loop_moments(h, cur));
    double d = INFINITY;
    if (h->last_loop.size() == cur.size()) {
        d = 0.0;
        for (size_t i = 0; i < cur.size(); ++i) {
            const double x = std::fabs(cur[i] - h->last_loop[i]);
            d = (x != x) ? INFINITY : std::max(d, x);  // an undefined moment never counts as converged
        }
    }
    h->last_loop.swap(cur);
    *delta = d;
    return CTM_OK;
}

ctm_status ctm_corner_spectra(ctm_handle h, double* out_host) {
    if (!h || !out_host) return CTM_ERR_ARG;
    std::vector<double> s;
    CKS(spectra(h, s));
    std::memcpy(out_host, s.data(), s.size() * sizeof(double));
    return CTM_OK;
}

ctm_status ctm_rdm1(ctm_handle h, int site, double* rho_host) {
    if (!h || !rho_host || site < 0 || site > 3) return CTM_ERR_ARG;
    CKS(check_ready(h));
    std::vector<double> r;
    CKS(rdm1_dev(h, site, r));
    normalise_trace(r, h->d);
    std::memcpy(rho_host, r.data(), r.size() * sizeof(double));
    return CTM_OK;
}

ctm_status ctm_rdm2(ctm_handle h, int site, int dx, int dy, double* rho_host) {
    if (!h || !rho_host || site < 0 || site > 3 || std::abs(dx) + std::abs(dy) != 1) return CTM_ERR_ARG;
    CKS(check_ready(h));
    std::vector<double> r;
    CKS(rdm2_any(h, site, dx, dy, r));
    std::memcpy(rho_host, r.data(), r.size() * sizeof(double));
    return CTM_OK;
}

ctm_status ctm_measure1(ctm_handle h, int site, const double* op, double* value) {
    if (!h || !op || !value) return CTM_ERR_ARG;
    const int d = h->d;
    std::vector<double> r((size_t)d * d);
    CKS(ctm_rdm1(h, site, r.data()));
    double v = 0.0;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) v += op[a * d + b] * r[b * d + a];
    *value = v;
    return CTM_OK;
}

ctm_status ctm_measure2(ctm_handle h, int site, int dx, int dy, const double* op, double* value) {
    if (!h || !op || !value) return CTM_ERR_ARG;
    const int n = h->d * h->d;
    std::vector<double> r((size_t)n * n);
    CKS(ctm_rdm2(h, site, dx, dy, r.data()));
    double v = 0.0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) v += op[a * n + b] * r[b * n + a];
    *value = v;
    return CTM_OK;
}

ctm_status ctm_op_from_elements(int d0, int d1, int n, const int* idx, const double* re, double* op_out) {
    if (d0 < 1 || d1 < 1 || n < 0 || !op_out || (n > 0 && (!idx || !re))) return CTM_ERR_ARG;
    const int m = d0 * d1;
    for (int i = 0; i < m * m; ++i) op_out[i] = 0.0;
    for (int l = 0; l < n; ++l) {
        const int i0 = idx[4 * l], j0 = idx[4 * l + 1], i1 = idx[4 * l + 2], j1 = idx[4 * l + 3];
        if (i0 < 0 || i0 >= d0 || i1 < 0 || i1 >= d0 || j0 < 0 || j0 >= d1 || j1 < 0 || j1 >= d1) return CTM_ERR_ARG;
        op_out[(i1 * d1 + j1) * m + (i0 * d1 + j0)] += re[l];
    }
    return CTM_OK;
}

// ---------------------------------------------------------------------------
// kernel-level entry points
// ---------------------------------------------------------------------------
ctm_status ctm_dgemm(int transA, int transB, int M, int N, int K, double alpha, const double* A, int lda,
                     const double* B, int ldb, double beta, double* C, int ldc, void* stream) {
    if (M < 0 || N < 0 || K < 0 || (M && N && (!A || !B || !C))) return CTM_ERR_ARG;
    if (ctm::dgemm(transA != 0, transB != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                   (cudaStream_t)stream) != cudaSuccess) {
        g_err = "ctm_dgemm launch failed";
        return CTM_ERR_CUDA;
    }
    return CTM_OK;
}

ctm_status ctm_permute(const double* src, double* dst, int ndim, const int* dims, const int* perm_,
                       void* stream) {
    if (!src || !dst || !dims || !perm_ || ndim < 1 || ndim > 8) return CTM_ERR_ARG;
    int seen = 0;
    for (int a = 0; a < ndim; ++a) {
        if (perm_[a] < 0 || perm_[a] >= ndim || dims[a] < 0) return CTM_ERR_ARG;
        seen |= 1 << perm_[a];
    }
    if (seen != (1 << ndim) - 1) return CTM_ERR_ARG;
    if (ctm::permute(src, dst, ndim, dims, perm_, (cudaStream_t)stream) != cudaSuccess) {
        g_err = "ctm_permute launch failed";
        return CTM_ERR_CUDA;
    }
    return CTM_OK;
}

size_t ctm_qr_workspace_bytes(int N, int k) { return (N >= k && k > 0) ? qr_ws_bytes(N, k) : 0; }

ctm_status ctm_qr(const double* Y, int N, int k, double* Q, double* R, void* ws, void* stream) {
    if (!Y || !Q || !R || !ws || k <= 0 || N < k) return CTM_ERR_ARG;
    if (ctm::qr(Y, N, k, Q, R, ws, (cudaStream_t)stream) != cudaSuccess) {
        g_err = "ctm_qr launch failed";
        return CTM_ERR_CUDA;
    }
    return CTM_OK;
}

size_t ctm_svd_workspace_bytes(int k) { return (k > 0 && k <= 1024) ? svd_ws_bytes(k) : 0; }

ctm_status ctm_svd(const double* G, int k, double* U, double* S, double* V, void* ws, void* stream) {
    if (!G || !U || !S || !V || !ws || k <= 0 || k > 1024) return CTM_ERR_ARG;
    if (ctm::svd(G, k, U, S, V, ws, (cudaStream_t)stream) != cudaSuccess) {
        g_err = "ctm_svd launch failed";
        return CTM_ERR_CUDA;
    }
    return CTM_OK;
}

ctm_status ctm_svd_noalloc(const double* G, int k, double* U, double* S, double* V, void* stream) {
    if (!G || !U || !S || !V) return CTM_ERR_ARG;
    if (k <= 0 || k > ctm::svd_noalloc_max_k()) {
        g_err = "ctm_svd_noalloc: k must be in 1.." + std::to_string(ctm::svd_noalloc_max_k()) +
                " (size of the static scratch array)";
        return CTM_ERR_ARG;
    }
    const cudaError_t e = ctm::svd_noalloc(G, k, U, S, V, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        g_err = std::string("ctm_svd_noalloc: ") + cudaGetErrorString(e);
        return CTM_ERR_CUDA;
    }
    return CTM_OK;
}

size_t ctm_gemm_ozaki_workspace_bytes(int M, int N, int K, int slices) {
    if (M <= 0 || N <= 0 || K <= 0 || slices < 2 || slices > 6) return 0;
    return 256 + ctm::oz_split_bytes(M, K, slices) + ctm::oz_split_bytes(N, K, slices) +
           ctm::oz_gemm_ws_bytes(M, N, K, slices);
}

ctm_status ctm_gemm_ozaki(int transA, int transB, int M, int N, int K, double alpha, const double* A, int lda,
                          const double* B, int ldb, double beta, double* C, int ldc, int slices, void* ws,
                          void* stream) {
    if (M < 0 || N < 0 || K <= 0 || slices < 2 || slices > 6 || (M && N && (!A || !B || !C || !ws)))
        return CTM_ERR_ARG;
    if (!M || !N) return CTM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)ws;
    int* err = (int*)w;
    void* sa = w + 256;
    void* sb = (char*)sa + ctm::oz_split_bytes(M, K, slices);
    void* part = (char*)sb + ctm::oz_split_bytes(N, K, slices);
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = ctm::oz_split(A, M, K, transA ? 1 : lda, transA ? lda : 1, slices, sa, st);
    if (e == cudaSuccess) e = ctm::oz_split(B, N, K, transB ? ldb : 1, transB ? 1 : ldb, slices, sb, st);
    if (e == cudaSuccess)
        e = ctm::oz_gemm(M, N, K, slices, sa, sb, alpha, beta, C, ldc, part,
                         ctm::oz_gemm_ws_bytes(M, N, K, slices), err, st);
    if (e != cudaSuccess) {
        g_err = std::string("ctm_gemm_ozaki: ") + cudaGetErrorString(e);
        return CTM_ERR_CUDA;
    }
    return CTM_OK;
}

size_t ctm_gemm_split_workspace_bytes(int precision, int M, int N, int K) {
    const int mode = tc_mode_of(precision);
    if (M <= 0 || N <= 0 || K <= 0 || (mode != 1 && mode != 2)) return 0;
    const int s = mode == 1 ? 3 : 2;
    return 256 + tc_split_bytes(M, K, mode, s) + tc_split_bytes(N, K, mode, s) + ctm::oz_gemm_ws_bytes(M, N, K, s, mode);
}

ctm_status ctm_gemm_split(int precision, int transA, int transB, int M, int N, int K, double alpha, const double* A,
                          int lda, const double* B, int ldb, double beta, double* C, int ldc, void* ws, void* stream) {
    const int mode = tc_mode_of(precision);
    if ((mode != 1 && mode != 2) || M < 0 || N < 0 || K <= 0 || (M && N && (!A || !B || !C || !ws)))
        return CTM_ERR_ARG;
    if (!M || !N) return CTM_OK;
    const int s = mode == 1 ? 3 : 2;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)ws;
    int* err = (int*)w;
    void* sa = w + 256;
    void* sb = (char*)sa + tc_split_bytes(M, K, mode, s);
    void* part = (char*)sb + tc_split_bytes(N, K, mode, s);
    const OzView ar{1, {M, 1, 1, 1}, {transA ? 1 : lda, 0, 0, 0}}, ak{1, {K, 1, 1, 1}, {transA ? lda : 1, 0, 0, 0}};
    const OzView bn{1, {N, 1, 1, 1}, {transB ? ldb : 1, 0, 0, 0}}, bk{1, {K, 1, 1, 1}, {transB ? 1 : ldb, 0, 0, 0}};
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = mode == 2 ? ctm::oz_split_tf32(A, M, K, ar, ak, sa, st) : ctm::oz_split_view(A, M, K, ar, ak, s, sa, st);
    if (e == cudaSuccess)
        e = mode == 2 ? ctm::oz_split_tf32(B, N, K, bn, bk, sb, st) : ctm::oz_split_view(B, N, K, bn, bk, s, sb, st);
    if (e == cudaSuccess)
        e = ctm::oz_gemm(M, N, K, s, sa, sb, alpha, beta, C, ldc, part, ctm::oz_gemm_ws_bytes(M, N, K, s, mode), err,
                         st, mode);
    if (e != cudaSuccess) {
        g_err = std::string("ctm_gemm_split: ") + cudaGetErrorString(e);
        return CTM_ERR_CUDA;
    }
    return CTM_OK;
}

ctm_status ctm_correlation(ctm_handle h, const double* opA, const double* opB, int rmax, double* out_host) {
    if (!h || !opA || !opB || !out_host || rmax < 0 || rmax > CTM_CORRELATION_MAX_R) return CTM_ERR_ARG;
    return correlation(h, opA, opB, rmax, out_host);
}

ctm_status ctm_transfer_spectrum(ctm_handle h, int dir, int index, int nev, int block, int max_iter, double tol,
                                 double* out_host, int* iters, double* change) {
    if (!h || !out_host || (dir != 0 && dir != 1) || index < 0 || index > 1 || nev < 1 || max_iter < 1 ||
        !(tol >= 0.0))
        return CTM_ERR_ARG;
    const long long n = (long long)h->chi * h->N;
    if (block < nev || block > ctm::small_eig_max() || block > n) return CTM_ERR_ARG;
    return transfer_spectrum(h, dir, index, nev, block, max_iter, tol, out_host, iters, change);
}

ctm_status ctm_small_eig(const double* H, int m, int ldh, double period, double* out, int* status, void* stream) {
    if (!H || !out || m < 1 || m > ctm::small_eig_max() || ldh < m || !(period > 0.0)) return CTM_ERR_ARG;
    const cudaError_t e = ctm::small_eig(H, m, ldh, period, out, status, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        g_err = std::string("ctm_small_eig: ") + cudaGetErrorString(e);
        return CTM_ERR_CUDA;
    }
    return CTM_OK;
}

ctm_status ctm_profile_enable(ctm_handle h, int on) {
    if (!h) return CTM_ERR_ARG;
    prof_collect(h);
    h->prof = on != 0;
    return CTM_OK;
}

ctm_status ctm_profile_read(ctm_handle h, ctm_profile_data* out, int reset) {
    if (!h || !out) return CTM_ERR_ARG;
    prof_collect(h);
    for (int c = 0; c < 8; ++c) {
        out->ms[c] = h->p_ms[c];
        out->flops[c] = h->p_flops[c];
        out->bytes[c] = h->p_bytes[c];
        out->calls[c] = h->p_calls[c];
        if (reset) h->p_ms[c] = h->p_flops[c] = h->p_bytes[c] = 0, h->p_calls[c] = 0;
    }
    if (reset) h->tags.clear();
    return CTM_OK;
}

long long ctm_kernel_launches(void) { return ctm::g_launches; }

ctm_status ctm_log_norm_per_site(ctm_handle h, double* lnkappa) {
    if (!h || !lnkappa) return CTM_ERR_ARG;
    CKS(check_ready(h));
    CKS(log_norm_per_site(h, lnkappa));
    return read_flag(h);
}

ctm_status ctm_init_env_random(ctm_handle h, uint64_t seed) {
    if (!h) return CTM_ERR_ARG;
    const size_t nC = (size_t)h->chi * h->chi, nT = (size_t)h->chi * h->D * h->D * h->chi;
    for (int w = 0; w < 8; ++w) {
        const size_t n = (w & 1) ? nT : nC;
        CK(ctm::rng_normal(h->env[0][w], n, seed, 0x454e56ull * 16 + (uint64_t)w, h->stream));
        if (w & 1) CK(ctm::sym_kk(h->env[0][w], h->chi, h->D, h->stream));
        for (int i = 1; i < 4; ++i)
            CK(cudaMemcpyAsync(h->env[i][w], h->env[0][w], n * sizeof(double), cudaMemcpyDeviceToDevice,
                               h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    h->env_set = 0xffffffffu;
    for (bool& w : h->warm_valid) w = false;
    for (auto& c : h->ozc) c.valid = false;
    return CTM_OK;
}

ctm_status ctm_fp64_peak(double* tflops) {
    if (!tflops) return CTM_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        g_err = "ctm_fp64_peak: no device";
        return CTM_ERR_CUDA;
    }
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    double* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double) * blocks * threads);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first launch warms up
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = ctm::dfma_probe(out, blocks, threads, iters, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0) best = std::min(best, ms);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        g_err = std::string("ctm_fp64_peak: ") + cudaGetErrorString(e);
        return CTM_ERR_CUDA;
    }
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
    return CTM_OK;
}

ctm_status ctm_wait_probe(long long limit_cycles, int arrive, int* flag_dev, void* stream) {
    if (!flag_dev || limit_cycles <= 0 || limit_cycles > 4000000000ll) return CTM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int f = 0;
    cudaError_t e = cudaMemsetAsync(flag_dev, 0, sizeof(int), st);
    if (e == cudaSuccess) e = ctm::wait_probe(limit_cycles, arrive, flag_dev, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&f, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        g_err = std::string("ctm_wait_probe: ") + cudaGetErrorString(e);
        return CTM_ERR_CUDA;
    }
    if (f) {
        g_err = "ctm_wait_probe: the bounded wait gave up";
        return CTM_ERR_TIMEOUT;
    }
    return CTM_OK;
}

ctm_status ctm_profile_report(ctm_handle h, char* buf, size_t len, int reset) {
    if (!h || !buf || len == 0) return CTM_ERR_ARG;
    prof_collect(h);
    std::string out = "{";
    bool first = true;
    char tmp[256];
    for (const auto& kv : h->tags) {
        snprintf(tmp, sizeof(tmp),
                 "%s\"%s\": {\"ms\": %.4f, \"calls\": %lld, \"launches\": %lld, \"flops\": %.6g, \"bytes\": %.6g}",
                 first ? "" : ", ", kv.first.c_str(), kv.second.ms, kv.second.calls, kv.second.launches,
                 kv.second.flops, kv.second.bytes);
        out += tmp;
        first = false;
    }
    out += "}";
    if (reset) h->tags.clear();
    if (out.size() + 1 > len) return CTM_ERR_ARG;
    memcpy(buf, out.c_str(), out.size() + 1);
    return CTM_OK;
}

}  // extern "C"
