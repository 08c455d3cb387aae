// Device-side data structures and the FP32 receiver-metric lattice.
//
// Notation (paper Sec. II): a frame has N symbols of n bits, tau = nN bits sent,
// rho bits received.  Drift states m in [-xmax, xmax] are indexed s = m + xmax,
// M = 2 xmax + 1 of them.  The drift change over one symbol is delta in
// [-n, nI]; j = n + delta in [0, n(I+1)] is the received length of one
// symbol, MN = n(I+1) + 1 values.  p = n i + m' is the received position where
// symbol i starts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mdk {

// chain_flags
constexpr int CH_SEGMENTED = 1;   // start/end rows and controller state come from ckpt/bedge/cst
constexpr int CH_REPLAY = 2;      // forward chain replays the recorded tilts (recompute sweep)

// test_flags
constexpr int TEST_SKIP_FIRST_COPY = 1;  // a recursion's first copy is never issued

constexpr int kMaxI = 7;        // insertion cap supported by the kernels
constexpr int kMaxMN = 64;      // n(I+1) + 1 <= 64 (received window fits 64 bits)
constexpr int kThreads = 256;   // producer block size
constexpr int kPsMaxQ = 256;    // codewords per symbol of the per-symbol-codebook producers

// Status codes shared with the C ABI (mapdec.h).
enum : int {
    ST_OK = 0, ST_ARG = 1, ST_DRIFT = 2, ST_ZERO = 3, ST_NOMEM = 4, ST_CUDA = 5,
    ST_TIMEOUT = 6, ST_UNSUPPORTED = 7
};

// Chain state carried between the segment launches of a frame (segmented mode).
struct ChainState {
    double theta, mean, logZ, lc_sum, lrow;
    int lc_cnt;
    int pad;
    long long steps;
};

// One frame as the kernels see it.  All pointers are device pointers.
struct FrameDev {
    // shape
    int q, n, N, I, xmax;
    int M;        // 2 xmax + 1 drift states
    int Mp;       // M rounded up to a multiple of 4 (row stride of alpha/beta)
    int MN;       // n(I+1) + 1 received lengths per symbol
    int MNS;      // row stride of W (odd, >= MN: bank-conflict-free smem rows)
    int P;        // received positions per APP-producer sub-tile
    int S;        // max symbols touched by one sub-tile
    int T;        // sub-tiles in this frame: ceil((rho+1)/P)
    int Pf;       // received positions per forward-producer tile (P unless the
                  // tensor-core forward producer picked its own)
    int Sf;       // max symbols touched by one forward tile
    int Tf;       // forward tiles: ceil((rho+1)/Pf)
    int ps;       // 1: one codebook per symbol (cw holds N*q words, C_i(D) at i*q + D);
                  // the producers are the per-symbol kernels, work item = i*psT + chunk
    int psC;      // per-symbol producers: start states per work item
    int psT;      // per-symbol producers: work items per symbol, ceil(M / psC)
    int Pgroups;  // tensor-core forward producer: 8-row groups of Pbuf
    unsigned char *Pbuf;  // the priors split into three bf16 pieces in that
                          // producer's operand layout (k_prior_split), or null
    // Stream decoding: drift priors of the frame's start and end (M floats each,
    // index m + xmax) replacing alpha_0 = [m = 0] and beta_N = [m = rho - tau];
    // null for an isolated frame.
    const float *phi0, *phiN;
    int nsub;     // sub-tiles per backward super-tile
    int S2;       // max symbols touched by one super-tile (rows of Lp per super-tile)
    int T2;       // backward super-tiles: ceil(T / nsub)
    int chainCD;  // destination/source states per chain chunk
    int chainStages;  // chunks in flight (ring of bulk-copy stages), <= 8
    uint32_t wait_limit;  // polls before a recursion's wait on a copy gives up (ST_TIMEOUT)
    int test_flags;       // TEST_SKIP_FIRST_COPY: the first copy is never issued (tests the timeout path)
    long long rho;
    long long wblk;  // floats per symbol block of W (M * MNS rounded up to 4)
    // FP32 lattice constants.  Every received bit carries a weight kappa: the
    // lattice runs with w' = kappa Pi/2 and Q' = kappa Q, so it yields
    // R~(y|x) = kappa^|y| R(y|x) exactly (kappa is a power of two).  The factor
    // is common to every term of a symbol's APP sum and shifts log P(Y) by
    // rho log kappa; it keeps FP32 forward/backward rows within range.
    float wpow[kMaxI + 1];   // w'^a
    float wder[kMaxI + 1];   // a w'^(a-1)  (d/dw' of wpow)
    float Pd, qsame, qdiff;  // Pd, kappa Pt (1-Ps), kappa Pt Ps
    // FP64 channel values for the log-likelihood and the gradient combination
    double dPi, dPd, dPs, dPt;
    double kappa, logk;      // received-bit weight and its log
    // inputs
    const uint32_t *rxbits;  // rho bits, bit b of word w = rx[32 w + b]; padded
    const uint32_t *cw;      // q codewords, bit r = x_{r+1}
    const float *priors;     // N*q
    // scratch
    float *W;        // N * wblk: W_i(s', j) = sum_D prior_i(D) R[p][D][j] at i*wblk + s'*MNS + j
    float *alpha;    // (N+1) * Mp normalised forward rows
    float *beta;     // (N+1) * Mp normalised backward rows
    float *Lp;       // T2 * S2 * q  partial unnormalised APP sums per super-tile
    float *Gp;       // T2 * S2 * 3  partial tangent sums per super-tile (gradient mode)
    float *Rout;     // receiver-metric dump (debug entry), (rho+1)*q*MN or null
    float *Rg;       // stored receiver metrics (or null: recompute), T * P*MN * DS:
                     // tile t at t*P*MN*DS, row pl*MN + j, column D (DS = roundup4(q))
    // Exponential tilt of the stored forward/backward rows (see k_chain):
    // thf[i], mcf[i]: tilt and mean drift of forward row i; thb[i]: tilt of
    // backward row i.  N+1 doubles each.
    double *thf, *mcf, *thb;
    double *Gc;      // per finalize chunk: 3 gradient partial sums (gradient mode)
    // Segments.  A descriptor covers the symbols [seg_i0, seg_i1); W, alpha,
    // beta, Lp and Gp point at buffers sized for that range, with base pointers
    // shifted so that absolute indices land in them.  The whole frame is one
    // segment (0, N) outside the segmented mode.
    int seg_i0, seg_i1;
    int fin_base;    // finalize chunk index of this segment's first chunk
    int fin_total;   // finalize chunks of the whole frame (gradient reduction)
    int chain_flags; // CH_* below
    float *ckpt;     // forward checkpoint rows (segmented mode): row s at s*Mp
    float *bedge;    // backward boundary row carried between segments (Mp floats)
    ChainState *cst; // [0] forward, [1] backward (segmented mode)
    // outputs
    float *app;      // N*q
    float *dpriors;  // N*q or null
    float *ext;      // N*q extrinsic outputs, or null
    double *loglik;  // 1
    double *dchan;   // 3 or null
    int *status;     // 1
};

// Work item of a producer launch: (frame, tile).
struct Work { int frame; int tile; };

__host__ __device__ inline long long floordiv(long long a, long long b) {
    long long d = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? d - 1 : d;
}
__host__ __device__ inline long long ceildiv(long long a, long long b) {
    return -floordiv(-a, b);
}

// Symbols i with |p - n i| <= xmax for some received position p in [p0, p1].
__host__ __device__ inline void range_symbols(const FrameDev &f, long long p0, long long p1,
                                              int &ilo, int &ihi) {
    if (p1 > f.rho) p1 = f.rho;
    long long lo = ceildiv(p0 - f.xmax, f.n);
    long long hi = floordiv(p1 + f.xmax, f.n);
    if (lo < f.seg_i0) lo = f.seg_i0;
    if (hi > f.seg_i1 - 1) hi = f.seg_i1 - 1;
    ilo = (int)lo;
    ihi = (int)hi;
}
// Forward tile t covers positions [t Pf, t Pf + Pf - 1].
__host__ __device__ inline void tile_symbols(const FrameDev &f, int tile, int &ilo, int &ihi) {
    const long long p0 = (long long)tile * f.Pf;
    range_symbols(f, p0, p0 + f.Pf - 1, ilo, ihi);
}
// Backward super-tile t covers positions [t P nsub, (t+1) P nsub - 1].
__host__ __device__ inline void super_symbols(const FrameDev &f, int tile, int &ilo, int &ihi) {
    const long long p0 = (long long)tile * f.P * f.nsub;
    range_symbols(f, p0, p0 + (long long)f.P * f.nsub - 1, ilo, ihi);
}

// 64 received bits starting at position p: bit k = y_{k+1} = Y[p + k].
__device__ __forceinline__ uint64_t rx_window(const uint32_t *__restrict__ rxb, long long p) {
    const long long w = p >> 5;
    const unsigned sh = (unsigned)(p & 31);
    const uint32_t a = __ldg(rxb + w), b = __ldg(rxb + w + 1), c = __ldg(rxb + w + 2);
    const uint32_t lo = __funnelshift_r(a, b, sh);
    const uint32_t hi = __funnelshift_r(b, c, sh);
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

// ---------------------------------------------------------------------------
// Receiver metric lattice, eqs. (F), (F_lastrow), FP32, fully unrolled for
// compile-time (n, I).  Row r holds F_{r, j}: arrived at row r by a vertical
// or diagonal step.  Row r+1 is built in place, column j descending:
//   G_{r,j}   = sum_{a=0}^{I} (Pi/2)^a F_{r, j-a}          (insertion run)
//   F_{r+1,j} = Pd G_{r,j} + Qdot(y_j | x_{r+1}) G_{r,j-1}
// G_{r,j-1} computed at column j is carried to column j-1.  Row r is non-zero
// only for j <= r(I+1), so every bound below folds at compile time.
// On return F[j] = R(y_1..y_j | x), j = 0..n(I+1).
//
// Tangent variants carry one extra row T = dF/dtheta for
//   MODE 1: theta = w = Pi/2,  MODE 2: theta = Pd,  MODE 3: theta = Pt Ps.
// ---------------------------------------------------------------------------
template <int NB, int IB, int MODE>
__device__ __forceinline__ void lattice_unrolled(uint32_t x, uint64_t y, const float *wpow,
                                                 const float *wder, float Pd, float qsame,
                                                 float qdiff, float (&F)[NB * (IB + 1) + 1],
                                                 float (&T)[NB * (IB + 1) + 1]) {
    constexpr int WW = NB * (IB + 1);
    float wp[IB + 1], wd[IB + 1];
#pragma unroll
    for (int a = 0; a <= IB; ++a) { wp[a] = wpow[a]; wd[a] = wder[a]; }
    // Received bits as all-ones / all-zeros masks.  Per row the pair (A, B) =
    // (Qdot for y = 0, Qdot for y = 1) is swapped by x_{r+1}; per node the
    // weight is picked exactly with one bitwise select, (A & ~m_j) | (B & m_j).
    uint32_t ym[WW];
#pragma unroll
    for (int j = 0; j < WW; ++j) ym[j] = 0u - (uint32_t)((y >> j) & 1u);
    const uint32_t qs_bits = __float_as_uint(qsame), qd_bits = __float_as_uint(qdiff);
#pragma unroll
    for (int j = 0; j <= WW; ++j) { F[j] = 0.f; if (MODE) T[j] = 0.f; }
    F[0] = 1.f;
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        const int hiF = r * (IB + 1);        // last non-zero column of row r
        const int hiN = (r + 1) * (IB + 1);  // last non-zero column of row r+1
        const uint32_t xm = 0u - ((x >> r) & 1u);            // x_{r+1} as a mask
        const uint32_t qa = (qs_bits & ~xm) | (qd_bits & xm);  // Qdot(0 | x)
        const uint32_t qb = (qd_bits & ~xm) | (qs_bits & xm);  // Qdot(1 | x)
        float gcar = 0.f, tcar = 0.f;        // G_{r,j}, TG_{r,j} at the current column
#pragma unroll
        for (int j = WW; j >= 0; --j) {
            if (j <= hiN) {
                float gprev = 0.f, tprev = 0.f;  // G_{r,j-1}, TG_{r,j-1}
                if (j >= 1) {
#pragma unroll
                    for (int a = 0; a <= IB; ++a) {
                        const int k = j - 1 - a;
                        if (k >= 0 && k <= hiF) {
                            gprev = (a == 0) ? F[k] : fmaf(wp[a], F[k], gprev);
                            if (MODE) {
                                tprev = (a == 0) ? T[k] : fmaf(wp[a], T[k], tprev);
                                if (MODE == 1 && a >= 1) tprev = fmaf(wd[a], F[k], tprev);
                            }
                        }
                    }
                }
                float f = Pd * gcar;
                float Q = 0.f;
                const uint32_t m = (j >= 1) ? ym[j >= 1 ? j - 1 : 0] : 0u;
                if (j >= 1) {
                    Q = __uint_as_float((qa & ~m) | (qb & m));
                    f = fmaf(Q, gprev, f);
                }
                if (MODE) {
                    float t = Pd * tcar;
                    if (j >= 1) t = fmaf(Q, tprev, t);
                    if (MODE == 2) t += gcar;
                    // substitution tangent: + G_{r,j-1} where y_j != x_{r+1}
                    if (MODE == 3 && j >= 1) t += __uint_as_float(__float_as_uint(gprev) & (m ^ xm));
                    T[j] = t;
                    tcar = tprev;
                }
                F[j] = f;
                gcar = gprev;
            }
        }
    }
}

// Same lattice with run-time n, I (any n(I+1) <= 63); rows live in local memory.
template <int MODE>
__device__ __noinline__ void lattice_runtime(int n, int I, uint32_t x, uint64_t y,
                                             const float *wpow, const float *wder, float Pd,
                                             float qsame, float qdiff, float *F, float *T) {
    const int WW = n * (I + 1);
    for (int j = 0; j <= WW; ++j) { F[j] = 0.f; if (MODE) T[j] = 0.f; }
    F[0] = 1.f;
    for (int r = 0; r < n; ++r) {
        const int hiF = r * (I + 1), hiN = (r + 1) * (I + 1);
        const uint64_t mm = y ^ (((x >> r) & 1u) ? ~0ull : 0ull);
        float gcar = 0.f, tcar = 0.f;
        for (int j = hiN; j >= 0; --j) {
            float gprev = 0.f, tprev = 0.f;
            if (j >= 1) {
                for (int a = 0; a <= I; ++a) {
                    const int k = j - 1 - a;
                    if (k >= 0 && k <= hiF) {
                        gprev = (a == 0) ? F[k] : fmaf(wpow[a], F[k], gprev);
                        if (MODE) {
                            tprev = (a == 0) ? T[k] : fmaf(wpow[a], T[k], tprev);
                            if (MODE == 1 && a >= 1) tprev = fmaf(wder[a], F[k], tprev);
                        }
                    }
                }
            }
            const bool mis = (j >= 1) && ((mm >> (j >= 1 ? j - 1 : 0)) & 1ull);
            const float Q = mis ? qdiff : qsame;
            float f = Pd * gcar;
            if (j >= 1) f = fmaf(Q, gprev, f);
            if (MODE) {
                float t = Pd * tcar;
                if (j >= 1) t = fmaf(Q, tprev, t);
                if (MODE == 2) t += gcar;
                if (MODE == 3 && j >= 1) t += mis ? gprev : 0.f;
                T[j] = t;
                tcar = tprev;
            }
            F[j] = f;
            gcar = gprev;
        }
    }
}

// ---------------------------------------------------------------------------
// mbarrier + bulk-copy helpers (sm_90+ PTX), with bounded waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 1-D bulk copy global -> shared, completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// 2^e exactly, for e in [-126, 127] (built from the exponent bits).
__device__ __forceinline__ float pow2i(int e) { return __int_as_float((e + 127) << 23); }

// Error-free sum: a + b = s + e exactly (Knuth's TwoSum, round to nearest).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// 4-byte asynchronous copy global -> shared (no registers held while in flight).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(gmem)
                 : "memory");
}
// Wait until every cp.async this thread issued has landed.
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}
// Wait for phase `parity` of `bar` to complete; gives up after `limit` polls.
// Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace mdk
