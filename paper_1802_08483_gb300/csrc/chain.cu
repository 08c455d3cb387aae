// Sequential parts of the decoder and small helper kernels.
//
//   k_pack     : received bits (one per byte) -> 32-bit words.
//   k_chain    : the forward recursion (eqs. alpha_prenorm, alpha_norm) or the
//                backward recursion (eq. beta, normalised by its sum) of one
//                frame, one CTA per (frame, direction).  The per-symbol
//                transition sums W_i(s', j) stream from global memory into
//                shared memory by 1-D bulk copies (cp.async.bulk) completed on
//                mbarriers, double-buffered, while the previous chunk is used.
//                Rows are kept exponentially tilted (see below) so that FP32
//                holds them; the forward chain keeps the exact FP64 record of
//                every normaliser and tilt and writes log P(Y).
//   k_finalize : APPs (eq. L, normalised over D), extrinsic outputs (eq. L
//                without the symbol's own prior), d logP / d prior and the
//                FP64 reduction of the channel-parameter gradient
//                (k_grad_reduce adds the chunks of a frame in order).
#include <cstdlib>

#include "mapdec_dev.cuh"
#include "mapdec_kernels.h"

namespace mdk {

// ---------------------------------------------------------------------------
__global__ void k_pack(const FrameDev *__restrict__ frames, const uint8_t *const *rx_bytes,
                       uint32_t *const *rx_words, int nframes) {
    const int fi = blockIdx.y;
    if (fi >= nframes) return;
    const long long rho = frames[fi].rho;
    const uint8_t *src = rx_bytes[fi];
    uint32_t *dst = rx_words[fi];
    const long long nwords = (rho + 31) / 32 + 3;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
         w += (long long)gridDim.x * blockDim.x) {
        uint32_t v = 0;
        const long long b0 = w * 32;
        for (int b = 0; b < 32; ++b) {
            const long long k = b0 + b;
            if (k < rho && src[k]) v |= (1u << b);
        }
        dst[w] = v;
    }
}

// ---------------------------------------------------------------------------
constexpr int kChainMaxThreads = 512;
constexpr int kChainThreads = 256;  // default block size
constexpr int kMaxStages = 8;

// Two FP32 sums at once (row sum and first moment); every thread gets the
// same result (the warps' partials are added in one fixed order).
__device__ __forceinline__ void block_sum2(float a, float b, float &sa, float &sb, float *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) { red[warp] = a; red[32 + warp] = b; }
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    float x = 0.f, y = 0.f;
    for (int w = 0; w < nw; ++w) { x += red[w]; y += red[32 + w]; }
    sa = x;
    sb = y;
}

// Tilt controller (see k_chain).
constexpr float kTiltGainMin = 0.02f;  // long-run smoothing of the entropy-rate estimate
constexpr float kTiltStepMax = 0.02f;  // largest change of the tilt between two rows
constexpr float kTiltMin = 0.2f, kTiltMax = 1.6f;
constexpr int kTiltEvery = 4;    // steps between tilt updates once settled
constexpr int kTiltSettle = 64;  // updates every step for the first steps

// Geometry of chunk k of a step: the same for every symbol, relative to the
// symbol's block of W (blocks are 16-byte aligned, so the aligned copy start,
// the shift to row r0 and the copy size do not depend on the symbol).
constexpr int kMaxChunks = 64;
struct ChunkTab {
    int d0[kMaxChunks], d1[kMaxChunks];  // owned states (alpha: destinations, beta: sources)
    int r0[kMaxChunks], r1[kMaxChunks];  // W rows staged
    int shift[kMaxChunks];               // floats between the aligned copy start and row r0
    int off[kMaxChunks];                 // aligned copy start within the symbol's block (floats)
    uint32_t bytes[kMaxChunks];          // copy size
};

__device__ __forceinline__ void chunk_geom(const FrameDev &f, int dir, int k, ChunkTab &t) {
    const int CD = f.chainCD, M = f.M;
    const int d0 = k * CD, d1 = min(M, d0 + CD);
    int r0, r1;
    if (dir == 0) {  // destination s gets sources s - nI .. s + n
        r0 = max(0, d0 - f.n * f.I);
        r1 = min(M, d1 + f.n);
    } else {
        r0 = d0;
        r1 = d1;
    }
    const int o0 = r0 * f.MNS, o1 = r1 * f.MNS;
    const int a0 = o0 & ~3, a1 = (o1 + 3) & ~3;
    t.d0[k] = d0;
    t.d1[k] = d1;
    t.r0[k] = r0;
    t.r1[k] = r1;
    t.shift[k] = o0 - a0;
    t.off[k] = a0;
    t.bytes[k] = a1 > a0 ? (uint32_t)(a1 - a0) * 4u : 16u;
}

// Exponential tilt.  The forward metric alpha_i(m) is the joint probability of
// a received prefix of L = n i + m bits, so a row falls off roughly like
// 2^{-h L} (h: entropy rate of the received bits) on top of the drift
// posterior; the backward metric rises the same way.  Far apart in FP32, the
// entries that carry the posterior would underflow.  The chains therefore store
//   alpha^_i(m) = alpha_i(m) 2^{theta_i L} / Z_i,   beta^_i(m) = beta_i(m) 2^{-theta'_i L} / Y_i
// with tilts theta driven toward h by the row sums: with a tilt theta a step
// grows the row sum by about 2^{(theta - h) n}, so theta_{i+1} = theta_i -
// g log2(growth) / n (g = 1/(steps+1), floored at kTiltGainMin); after the
// first kTiltSettle steps it is updated every kTiltEvery steps from the mean
// growth of the steps since.  The producers already weight every received bit
// by 2 (theta = 1), so a step multiplies the transition sums by
// 2^{(theta - 1) j} (j = received length) and pre-scales the source row by
// 2^{(theta_{i+1} - theta_i)(m - mean)}.  Each new row is divided by the
// power of two 2^e just below its sum c (exact; the row then sums to [1, 2)),
// so Z_i is a power of two times the tilt factors, kept exactly in FP64, and
// log P(Y) = log alpha^_N(rho - tau) + log Z_N - theta_N rho log 2.  The APP
// producer applies the matching exact factor; the per-row constants cancel in
// the APPs and in the gradient.
//
// The W rows of a step stream into shared memory in chunks of chainCD states
// (plus the band halo in the forward direction) by 1-D bulk copies completed
// on mbarriers, chainStages chunks in flight; every wait is bounded.
__global__ void __launch_bounds__(kChainMaxThreads) k_chain(const FrameDev *__restrict__ frames,
                                                         const Work *__restrict__ work) {
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    const int dir = wk.tile & 1;  // 0 = forward (alpha), 1 = backward (beta); bit 1: replay
    const int M = f.M, Mp = f.Mp, MNS = f.MNS, MN = f.MN, n = f.n, N = f.N, xmax = f.xmax;
    const long long rho = f.rho;
    const int CD = f.chainCD;
    const int nck = (M + CD - 1) / CD;
    const int NST = f.chainStages;
    const int i0 = f.seg_i0, i1 = f.seg_i1;  // symbols of this launch (segment)
    const int send = (int)(rho - (long long)n * N) + xmax;  // state of the end drift
    const bool segm = (f.chain_flags & CH_SEGMENTED) != 0;
    const bool replay = dir == 0 && (wk.tile & 2) != 0;
    // first launch of this direction: the frame boundary; otherwise the row carried over
    const bool fresh = dir == 0 ? (i0 == 0) : (i1 == N);

    __shared__ uint64_t bar[kMaxStages];
    __shared__ float red[64];
    __shared__ int s_fail;
    __shared__ float s_th[3];  // tilt of the current row, of the row being built, row mean
    __shared__ float vfac[kMaxMN];
    extern __shared__ float4 sm4[];
    float *cur = reinterpret_cast<float *>(sm4);
    float *nxt = cur + Mp;
    float *stage0 = nxt + Mp;
    const size_t stageFloats = ((size_t)(CD + MN + 1) * MNS + 8 + 3) & ~(size_t)3;

    for (int s = threadIdx.x; s < Mp; s += blockDim.x) {
        float v;
        if (fresh) v = (s == (dir == 0 ? xmax : send)) ? 1.f : 0.f;
        else v = (dir == 0) ? f.ckpt[s] : f.bedge[s];
        cur[s] = v;
        nxt[s] = 0.f;
    }
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int st = 0; st < NST; ++st) mbar_init(&bar[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // Stream decoding: a boundary drift prior replaces the point mass
    // (alpha_0 = phi0, beta_N = phiN; Sec. II-C).  In the tilted rows the start
    // row is alpha^_0(m) = phi0(m) 2^m / Z_0 (tilt 1, received length m) and the
    // end row beta^_N(m) is proportional to phiN(m) 2^-m; both are first scaled
    // by 2^-emax (emax the largest exponent over the prior's support, exact),
    // then divided by the power of two below their sum like every row, and
    // log2 Z_0 = emax + that exponent starts the forward record.
    const float *prior = !fresh ? nullptr : (dir == 0 ? f.phi0 : f.phiN);
    __shared__ int s_emax;
    long long zexp0 = 0;  // log2 Z_0 of a prior start row (forward)
    float mean0 = (dir == 0) ? 0.f : (float)(send - xmax);
    if (prior) {
        if (threadIdx.x == 0) s_emax = -(1 << 30);
        __syncthreads();
        for (int s = threadIdx.x; s < M; s += blockDim.x)
            if (prior[s] > 0.f) atomicMax(&s_emax, dir == 0 ? s - xmax : xmax - s);
        __syncthreads();
        const int emax = s_emax;
        float part0 = 0.f, partm0 = 0.f;
        for (int s = threadIdx.x; s < M; s += blockDim.x) {
            const float w = prior[s];
            const int e = (dir == 0 ? s - xmax : xmax - s) - emax;  // <= 0
            const float v = (w > 0.f && e > -150) ? ldexpf(w, e) : 0.f;
            cur[s] = v;
            part0 += v;
            partm0 = fmaf(v, (float)(s - xmax), partm0);
        }
        float c0, cm0;
        block_sum2(part0, partm0, c0, cm0, red);
        if (!(c0 > 0.f)) {  // no mass inside the drift limits (same in every thread)
            if (threadIdx.x == 0) atomicMax(f.status, ST_ZERO);
            return;         // nothing issued yet
        }
        int ex;
        frexpf(c0, &ex);
        const float inv = ldexpf(1.f, 1 - ex);
        for (int s = threadIdx.x; s < M; s += blockDim.x) cur[s] *= inv;
        zexp0 = (long long)emax + ex - 1;
        mean0 = cm0 / c0;
        __syncthreads();
    }
    {
        float *row0 = (dir == 0) ? f.alpha + (size_t)i0 * Mp : f.beta + (size_t)i1 * Mp;
        for (int s = threadIdx.x; s < Mp; s += blockDim.x) row0[s] = cur[s];
    }
    auto symbol_of = [&](int st) { return dir == 0 ? i0 + st : i1 - 1 - st; };
    // Chunk table, and a self-check of every copy it implies: source inside
    // this launch's symbols of W (plus the 16-float tail slack), destination
    // inside its stage, 16-byte alignment and size.  A violation records
    // ST_ARG and the chain does not start.
    __shared__ ChunkTab tab;
    for (int k = threadIdx.x; k < nck && k < kMaxChunks; k += blockDim.x) {
        chunk_geom(f, dir, k, tab);
        const bool ok = tab.off[k] + (long long)tab.bytes[k] / 4 <= f.wblk + 16 &&
                        tab.bytes[k] % 16 == 0 && tab.bytes[k] / 4 <= stageFloats;
        if (!ok) atomicExch(&s_fail, ST_ARG);
    }
    if (threadIdx.x == 0 && (nck > kMaxChunks || ((uintptr_t)f.W & 15) != 0 || (f.wblk & 3) != 0 ||
                             ((uintptr_t)stage0 & 15) != 0 || (stageFloats & 3) != 0))
        atomicExch(&s_fail, ST_ARG);
    __syncthreads();
    if (s_fail) {  // same in every thread (read after the barrier); nothing issued yet
        if (threadIdx.x == 0) atomicMax(f.status, s_fail);
        return;
    }
    const long long total = (long long)(i1 - i0) * nck;
    // thread 0's issue cursor: chunks issued so far, and the next one's place
    long long issued = 0;
    int is_st = 0, is_k = 0, is_slot = 0;
    auto issue_next = [&]() {
        const float *src = f.W + (size_t)symbol_of(is_st) * f.wblk + tab.off[is_k];
        uint64_t *b = &bar[is_slot];
        if (!((f.test_flags & TEST_SKIP_FIRST_COPY) && issued == 0)) {
            mbar_expect_tx(b, tab.bytes[is_k]);
            bulk_g2s(stage0 + (size_t)is_slot * stageFloats, src, tab.bytes[is_k], b);
        }
        ++issued;
        if (++is_k == nck) { is_k = 0; ++is_st; }
        if (++is_slot == NST) is_slot = 0;
    };
    if (threadIdx.x == 0)
        while (issued < NST && issued < total) issue_next();

    // controller state (thread 0); log2 Z as an integer sum of the row
    // scalings plus the FP64 sum of the tilt terms (changed rows only)
    long long zexp = zexp0;
    double ztilt = 0.0;
    float theta = 1.f;   // tilt of the current row
    float mean = mean0;  // its mean drift
    float lrow = 0.f;      // log2 of the current row's sum
    float lc_prev = 0.f;   // sum of log2 growth since the last tilt update
    int lc_cnt = 0;        // number of steps in lc_prev
    int steps = 0;         // every thread: steps taken in this direction so far
    if (!fresh && segm) {
        const ChainState &cs = f.cst[dir];
        steps = (int)cs.steps;
        if (threadIdx.x == 0) {
            theta = (float)cs.theta;
            mean = (float)cs.mean;
            ztilt = cs.logZ / 0.6931471805599453;
            lc_prev = (float)cs.lc_sum;
            lrow = (float)cs.lrow;
            lc_cnt = cs.lc_cnt;
        }
    }
    if (replay) steps = i0;
    if (threadIdx.x == 0 && fresh && !replay) {
        if (dir == 0) { f.thf[0] = 1.0; f.mcf[0] = (double)mean0; }
        else f.thb[N] = 1.0;
    }
    // this thread's share of the row sum and of its first moment
    float part = 0.f, partm = 0.f;
    float th_cur = 1.f, th_new = 1.f, mc = 0.f;
    if (!fresh && segm && !replay) {
        // continuing a recursion: the first step here need not be an update
        // step, so restore the row's tilt and its transition weights as the
        // previous launch left them
        if (threadIdx.x == 0) {
            s_th[0] = theta;
            s_th[2] = mean;
        }
        __syncthreads();
        th_cur = th_new = s_th[0];
        mc = s_th[2];
        for (int j = threadIdx.x; j < MN; j += blockDim.x) vfac[j] = exp2f((th_cur - 1.f) * (float)j);
        __syncthreads();
    }
    bool failed = false;
    long long gfail = 0;
    int st = 0, k = 0, slot = 0;
    uint32_t ph = 0;
    for (long long g = 0; g < total; ++g) {
        const int i = symbol_of(st);
        const bool update = replay || steps < kTiltSettle || (steps & (kTiltEvery - 1)) == 0;
        if (k == 0 && update) {
            // start of an update step: choose the tilt of the rows from here on
            // (the recompute sweep replays the tilts recorded by the first sweep)
            if (threadIdx.x == 0 && replay) {
                s_th[0] = (float)f.thf[i];
                s_th[1] = (float)f.thf[i + 1];
                s_th[2] = (float)f.mcf[i];
            } else if (threadIdx.x == 0) {
                float tn = theta;
                if (steps > 0 && lc_cnt > 0) {
                    const float gain =
                        fminf(1.f, fmaxf(kTiltGainMin, (float)lc_cnt / (float)(steps + 1)));
                    const float d = fminf(kTiltStepMax,
                                          fmaxf(-kTiltStepMax, -gain * (lc_prev / (float)lc_cnt) / (float)n));
                    tn = fminf(kTiltMax, fmaxf(kTiltMin, theta + d));
                }
                s_th[0] = theta;
                s_th[1] = tn;
                s_th[2] = mean;
                lc_prev = 0.f;
                lc_cnt = 0;
            }
            __syncthreads();
            th_cur = s_th[0];
            th_new = s_th[1];
            mc = s_th[2];
            // forward: transition weight 2^{(theta_{i+1}-1) j}; backward: 2^{(theta'_{i+1}-1) j}
            const float phi = (dir == 0 ? th_new : th_cur) - 1.f;
            for (int j = threadIdx.x; j < MN; j += blockDim.x) vfac[j] = exp2f(phi * (float)j);
            if (dir == 0) {
                const float dth = th_new - th_cur;
                if (dth != 0.f)
                    for (int s = threadIdx.x; s < M; s += blockDim.x)
                        cur[s] *= exp2f(dth * ((float)(s - xmax) - mc));
            }
            __syncthreads();
        } else if (k == 0) {
            // no update: the row keeps its tilt (backward: the transition weight of
            // a step uses the source row's tilt, which is now th_new)
            if (dir == 1 && th_cur != th_new) {
                th_cur = th_new;
                const float phi = th_cur - 1.f;
                for (int j = threadIdx.x; j < MN; j += blockDim.x) vfac[j] = exp2f(phi * (float)j);
                __syncthreads();
            }
            th_cur = th_new;
        }
        const int cd0 = tab.d0[k], cd1 = tab.d1[k], cr0 = tab.r0[k], cr1 = tab.r1[k];
        const float *buf = stage0 + (size_t)slot * stageFloats + tab.shift[k];
        if (!mbar_wait(&bar[slot], ph, f.wait_limit)) atomicExch(&s_fail, ST_TIMEOUT);
        // valid source rows: window start p = n i + s - xmax inside [0, rho]
        const int vlo = max(0, xmax - n * i);
        const long long vhi_l = rho - (long long)n * i + xmax;
        const int vhi = (int)min((long long)M - 1, vhi_l);
        // JS lanes share one state, each summing every JS-th term with four
        // accumulators; the lanes combine by shuffles in a fixed order.
        const int nst = cd1 - cd0;
        int JS = 1;
        while (JS < 8 && nst * JS * 2 <= (int)blockDim.x) JS *= 2;
        const int lgJS = JS == 1 ? 0 : (JS == 2 ? 1 : (JS == 4 ? 2 : 3));
        const int lo = max(cr0, vlo), hi = min(cr1 - 1, vhi);
        for (int w0 = 0; w0 < nst * JS; w0 += blockDim.x) {
            const int w = w0 + (int)threadIdx.x;
            const int s = cd0 + (w >> lgJS), js = w & (JS - 1);
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            if (w < nst * JS) {
                if (dir == 0) {
                    // alpha'(s) = sum_j alpha(s - j + n) W[s - j + n][j] vfac[j]
                    const int jlo = max(0, s + n - hi), jhi = min(MN - 1, s + n - lo);
                    const float *cp = cur + (s + n);
                    const float *bp = buf + (size_t)(s + n - cr0) * MNS;
                    const int dm = MNS - 1;
                    int j = jlo + js;
                    for (; j + 3 * JS <= jhi; j += 4 * JS) {
                        const int j1 = j + JS, j2 = j + 2 * JS, j3 = j + 3 * JS;
                        a0 = fmaf(cp[-j], bp[-j * dm] * vfac[j], a0);
                        a1 = fmaf(cp[-j1], bp[-j1 * dm] * vfac[j1], a1);
                        a2 = fmaf(cp[-j2], bp[-j2 * dm] * vfac[j2], a2);
                        a3 = fmaf(cp[-j3], bp[-j3 * dm] * vfac[j3], a3);
                    }
                    for (; j <= jhi; j += JS) a0 = fmaf(cp[-j], bp[-j * dm] * vfac[j], a0);
                } else if (s >= vlo && s <= vhi) {
                    // beta'(s) = sum_j W[s][j] vfac[j] beta(s + j - n)
                    const int jlo = max(0, n - s), jhi = min(MN - 1, M - 1 - s + n);
                    const float *wr = buf + (size_t)(s - cr0) * MNS;
                    const float *cq = cur + (s - n);
                    int j = jlo + js;
                    for (; j + 3 * JS <= jhi; j += 4 * JS) {
                        const int j1 = j + JS, j2 = j + 2 * JS, j3 = j + 3 * JS;
                        a0 = fmaf(wr[j] * vfac[j], cq[j], a0);
                        a1 = fmaf(wr[j1] * vfac[j1], cq[j1], a1);
                        a2 = fmaf(wr[j2] * vfac[j2], cq[j2], a2);
                        a3 = fmaf(wr[j3] * vfac[j3], cq[j3], a3);
                    }
                    for (; j <= jhi; j += JS) a0 = fmaf(wr[j] * vfac[j], cq[j], a0);
                }
            }
            float acc = (a0 + a1) + (a2 + a3);
            for (int o = 1; o < JS; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (w < nst * JS && js == 0) {
                if (dir == 1) {
                    // post-scale 2^{(theta'_{i+1} - theta'_i)(m - mean)}
                    const float dth = th_cur - th_new;
                    if (dth != 0.f) acc *= exp2f(dth * ((float)(s - xmax) - mc));
                }
                nxt[s] = acc;
                part += acc;
                partm = fmaf(acc, (float)(s - xmax), partm);
            }
        }
        __syncthreads();  // stage consumed by everyone
        if (s_fail) {     // a wait gave up (written before the barrier: same in every thread)
            failed = true;
            gfail = g;    // chunks g .. issued-1 may still be in flight
            break;
        }
        if (threadIdx.x == 0 && issued < total) issue_next();
        if (k == nck - 1) {
            // end of a step: scale by a power of two, keep the exact record
            float c, cm;
            block_sum2(part, partm, c, cm, red);
            part = 0.f;
            partm = 0.f;
            const bool bad = !(c >= 1.2e-38f) || !(c <= 3.0e38f);  // same in every thread
            if (bad) {
                if (threadIdx.x == 0) s_fail = ST_ZERO;
                failed = true;
                gfail = g + 1;
                break;
            }
            int ex;
            frexpf(c, &ex);  // c = m 2^ex, m in [0.5, 1)
            const float inv = ldexpf(1.f, 1 - ex);
            if (threadIdx.x == 0) {
                const float lc = log2f(c);
                if (dir == 0 && !replay) {
                    zexp += ex - 1;
                    if (th_new != th_cur)
                        ztilt += (double)(th_new - th_cur) * ((double)n * i + (double)mc);
                    f.thf[i + 1] = (double)th_new;
                    f.mcf[i + 1] = (double)(cm / c);
                } else if (dir == 1) {
                    f.thb[i] = (double)th_new;
                }
                theta = th_new;
                mean = cm / c;
                lc_prev += lc - lrow;
                lrow = lc - (float)(ex - 1);
                ++lc_cnt;
            }
            ++steps;
            float *row = (dir == 0) ? f.alpha + (size_t)(i + 1) * Mp : f.beta + (size_t)i * Mp;
            for (int s = threadIdx.x; s < M; s += blockDim.x) {
                const float v = nxt[s] * inv;
                cur[s] = v;
                row[s] = v;
            }
            __syncthreads();
        }
        if (++k == nck) { k = 0; ++st; }
        if (++slot == NST) { slot = 0; ph ^= 1u; }
    }
    if (failed) {
        // Copies already issued (chunks gfail .. issued-1) must land before the
        // CTA's shared memory is released: wait for them, again with a bound.
        __syncthreads();
        if (threadIdx.x == 0) {
            for (long long h = gfail; h < issued; ++h)
                mbar_wait(&bar[h % NST], (uint32_t)((h / NST) & 1), f.wait_limit);
            atomicMax(f.status, s_fail);
        }
        __syncthreads();
        return;
    }
    if (segm && !replay) {
        // carry the boundary row and the controller state to the next launch
        float *edge = (dir == 0) ? f.ckpt + Mp : f.bedge;
        for (int s = threadIdx.x; s < Mp; s += blockDim.x) edge[s] = cur[s];
        if (threadIdx.x == 0) {
            ChainState &cs = f.cst[dir];
            cs.theta = theta;
            cs.mean = mean;
            cs.logZ = ((double)zexp + ztilt) * 0.6931471805599453;
            cs.lc_sum = lc_prev;
            cs.lrow = lrow;
            cs.lc_cnt = lc_cnt;
            cs.steps = steps;
        }
    }
    if (dir == 0 && !replay && i1 == N && threadIdx.x == 0) {
        if (f.phiN) {
            // log P = log Z_N - theta tau log 2 + log sum_m phiN(m) alpha^_N(m) 2^{-theta m},
            // the sum formed in FP64 relative to its largest term
            const double th = (double)theta;
            double lmax = -1e300;
            for (int s = 0; s < M; ++s)
                if (f.phiN[s] > 0.f && cur[s] > 0.f)
                    lmax = fmax(lmax, log2((double)cur[s]) + log2((double)f.phiN[s]) -
                                          th * (double)(s - xmax));
            double sum = 0.0;
            if (lmax > -1e300)
                for (int s = 0; s < M; ++s)
                    if (f.phiN[s] > 0.f && cur[s] > 0.f)
                        sum += exp2(log2((double)cur[s]) + log2((double)f.phiN[s]) -
                                    th * (double)(s - xmax) - lmax);
            if (!(sum > 0.0)) {
                atomicMax(f.status, ST_ZERO);
            } else {
                *f.loglik = (lmax + log2(sum) + (double)zexp + ztilt -
                             th * (double)((long long)n * N)) * 0.6931471805599453;
            }
        } else {
            const float aN = cur[send];
            if (!(aN > 0.f)) {
                atomicMax(f.status, ST_ZERO);
            } else {
                *f.loglik = log((double)aN) +
                            ((double)zexp + ztilt - (double)theta * (double)rho) * 0.6931471805599453;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Finalize: one CTA per (frame, chunk of kFinChunk symbols), one warp per
// symbol, lanes over D.  Gradient sums of a chunk go to Gc[chunk]; a second
// kernel adds the chunks of a frame in order (deterministic).
constexpr int kFinThreads = 256;
constexpr int kFinChunk = 64;

// Row of the APP partials of symbol i in super-tile tlo + t; the first 32 are
// cached one per lane (warp-uniform t), further ones are computed directly.
__device__ __forceinline__ long long lp_row(const FrameDev &f, long long myrow, int t, int tlo,
                                            int i) {
    const long long cached = __shfl_sync(0xffffffffu, myrow, t & 31);
    if (f.ps) return (long long)tlo + t;  // per-symbol producers: rows i*psT .. i*psT+psT-1
    if (t < 32) return cached;
    int ilo, ihi;
    super_symbols(f, tlo + t, ilo, ihi);
    return (long long)(tlo + t) * f.S2 + (i - ilo);
}

__global__ void __launch_bounds__(kFinThreads) k_finalize(const FrameDev *__restrict__ frames,
                                                          const Work *__restrict__ work,
                                                          int grad) {
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    __shared__ double red[3][32];
    if (*f.status != ST_OK) return;
    const int q = f.q, n = f.n, xmax = f.xmax;
    const long long P2 = (long long)f.P * f.nsub;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const double Pt = f.dPt, Ps = f.dPs, Pd = f.dPd, k = f.kappa;
    // the lattice ran with w' = k Pi/2, Q'm = k Pt (1-Ps), Q's = k Pt Ps
    const double Qm = k * Pt * (1.0 - Ps), Qs = k * Pt * Ps;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    bool bad = false;
    const int i0 = f.seg_i0 + (wk.tile - f.fin_base) * kFinChunk;
    const int i1 = min(f.seg_i1, i0 + kFinChunk);
    for (int i = i0 + warp; i < i1; i += nw) {
        long long plo = (long long)n * i - xmax, phi = (long long)n * i + xmax;
        if (plo < 0) plo = 0;
        if (phi > f.rho) phi = f.rho;
        int tlo = (int)(plo / P2), thi = (int)(phi / P2);
        if (f.ps) {  // one row per work item (symbol, chunk of start states)
            tlo = i * f.psT;
            thi = tlo + f.psT - 1;
        }
        // lane l holds the Lp row offset of super-tile tlo + l for this symbol
        long long myrow = 0;
        if (!f.ps && tlo + lane <= thi) {
            int ilo, ihi;
            super_symbols(f, tlo + lane, ilo, ihi);
            myrow = (long long)(tlo + lane) * f.S2 + (i - ilo);
        }
        double z = 0.0, zu = 0.0;
        // pass 1: unnormalised sums L^u(D) (eq. L without the prior) into app,
        // z = sum_D prior(D) L^u(D) and, for the extrinsic output, zu = sum_D L^u(D)
        for (int D0 = 0; D0 < q; D0 += 32) {
            const int D = D0 + lane;
            float s = 0.f;
            for (int t = 0; t <= thi - tlo; ++t) {
                const long long row = lp_row(f, myrow, t, tlo, i);
                if (D < q) s += f.Lp[row * q + D];
            }
            if (D < q) {
                f.app[(size_t)i * q + D] = s;
                z += (double)f.priors[(size_t)i * q + D] * (double)s;
                zu += (double)s;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            z += __shfl_xor_sync(0xffffffffu, z, o);
            zu += __shfl_xor_sync(0xffffffffu, zu, o);
        }
        if (!(z > 0.0)) { bad = true; continue; }
        const double iz = 1.0 / z;
        const double izu = 1.0 / zu;  // zu >= z / max prior > 0
        // pass 2: each lane rescales the entries it wrote
        for (int D = lane; D < q; D += 32) {
            const size_t e = (size_t)i * q + D;
            const double lu = (double)f.app[e];
            f.app[e] = (float)((double)f.priors[e] * lu * iz);
            if (f.dpriors) f.dpriors[e] = (float)(lu * iz);
            if (f.ext) f.ext[e] = (float)(lu * izu);
        }
        if (grad) {
            double Sw = 0.0, Sd = 0.0, Ss = 0.0;
            for (int t = 0; t <= thi - tlo; ++t) {
                const long long row = lp_row(f, myrow, t, tlo, i);
                const float *gp = f.Gp + row * 3;
                Sw += gp[0];
                Sd += gp[1];
                Ss += gp[2];
            }
            if (lane == 0) {
                // Sw, Sd, Ss: sums with dR~/dw', dR~/dPd, dR~/dQ's.  R~ is homogeneous
                // of degree n in (Pd, Q'm, Q's) (every bit is deleted or transmitted),
                // so Pd dR~/dPd + Q'm dR~/dQ'm + Q's dR~/dQ's = n R~ gives the Q'm sum.
                // Chain rule with w' = k Pi/2, Q'm = k Pt (1-Ps), Q's = k Pt Ps, Pt = 1-Pi-Pd.
                const double Sm = ((double)n * z - Pd * Sd - Qs * Ss) / Qm;
                g0 += (0.5 * k * Sw - k * (1.0 - Ps) * Sm - k * Ps * Ss) * iz;
                g1 += (Sd - k * (1.0 - Ps) * Sm - k * Ps * Ss) * iz;
                g2 += (-k * Pt * Sm + k * Pt * Ss) * iz;
            }
        }
    }
    if (bad && lane == 0) atomicMax(f.status, ST_ZERO);
    if (grad && f.Gc) {
        if (lane == 0) { red[0][warp] = g0; red[1][warp] = g1; red[2][warp] = g2; }
        __syncthreads();
        if (threadIdx.x < 3) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[threadIdx.x][w];
            f.Gc[(size_t)wk.tile * 3 + threadIdx.x] = s;
        }
    }
}

// Sums the chunk gradients of every frame in chunk order.
__global__ void k_grad_reduce(const FrameDev *__restrict__ frames, int nframes) {
    const int fi = blockIdx.x * blockDim.x + threadIdx.x;
    if (fi >= nframes) return;
    const FrameDev &f = frames[fi];
    if (!f.dchan || !f.Gc || *f.status != ST_OK) return;
    const int nch = f.fin_total;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int c = 0; c < nch; ++c) {
        s0 += f.Gc[3 * c];
        s1 += f.Gc[3 * c + 1];
        s2 += f.Gc[3 * c + 2];
    }
    f.dchan[0] = s0;
    f.dchan[1] = s1;
    f.dchan[2] = s2;
}

// ---------------------------------------------------------------------------
// Copies between pinned host memory and device memory by the SMs: 16 bytes per
// thread and step over a grid-stride loop, reading or writing the host side
// through its device mapping (NVLink-C2C).  Both pointers 16-byte aligned; n16
// 16-byte words.
__global__ void k_copy16(uint4 *__restrict__ dst, const uint4 *__restrict__ src, size_t n16) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n16; k += stride)
        dst[k] = src[k];
}

// ---------------------------------------------------------------------------
// Launch wrappers (host).
cudaError_t launch_copy16(void *dst, const void *src, size_t n16, int sms, cudaStream_t st) {
    if (n16 == 0) return cudaSuccess;
    const size_t per = 256;
    size_t blocks = (n16 + per - 1) / per;
    const size_t cap = (size_t)(sms > 0 ? sms : 152) * 4;
    if (blocks > cap) blocks = cap;
    k_copy16<<<(unsigned)blocks, (unsigned)per, 0, st>>>(static_cast<uint4 *>(dst),
                                                          static_cast<const uint4 *>(src), n16);
    return cudaGetLastError();
}

cudaError_t launch_pack(const FrameDev *frames, const uint8_t *const *rx_bytes,
                        uint32_t *const *rx_words, int nframes, long long max_words,
                        cudaStream_t st) {
    if (nframes <= 0) return cudaSuccess;
    int gx = (int)((max_words + 255) / 256);
    if (gx > 64) gx = 64;
    if (gx < 1) gx = 1;
    dim3 grid(gx, nframes);
    k_pack<<<grid, 256, 0, st>>>(frames, rx_bytes, rx_words, nframes);
    return cudaGetLastError();
}

size_t chain_smem_bytes(const FrameDev &f) {
    const size_t stageFloats = ((size_t)(f.chainCD + f.MN + 1) * f.MNS + 8 + 3) & ~(size_t)3;
    return 4 * (2 * (size_t)f.Mp + (size_t)f.chainStages * stageFloats);
}

cudaError_t launch_chain(const FrameDev *frames, const Work *work, int nwork, size_t smem,
                         int threads, cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    // Raise the opt-in limit to the device maximum, once per device (the
    // attribute is per device): graphs hold chain launches of several waves
    // with different sizes, and every one must stay valid.
    static std::atomic<int> max_dyn[64];  // 0 = not yet set on that device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int lim = (dev >= 0 && dev < 64) ? max_dyn[dev].load(std::memory_order_acquire) : 0;
    if (lim <= 0) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k_chain);
        if (e != cudaSuccess) return e;
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        lim = optin - (int)fa.sharedSizeBytes;
        e = cudaFuncSetAttribute(k_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) max_dyn[dev].store(lim, std::memory_order_release);
    }
    if ((long long)smem > lim) return cudaErrorInvalidValue;
    if (threads != 128 && threads != 256 && threads != 512) threads = kChainThreads;
    k_chain<<<nwork, threads, smem, st>>>(frames, work);
    return cudaGetLastError();
}

int finalize_chunks(int N) { return (N + kFinChunk - 1) / kFinChunk; }
size_t chain_state_bytes() { return sizeof(ChainState); }

cudaError_t launch_finalize(const FrameDev *frames, const Work *work, int nwork, int nframes,
                            int grad, cudaStream_t st, bool reduce) {
    if (nwork > 0) k_finalize<<<nwork, kFinThreads, 0, st>>>(frames, work, grad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !grad || !reduce || nframes <= 0) return e;
    k_grad_reduce<<<(nframes + 127) / 128, 128, 0, st>>>(frames, nframes);
    return cudaGetLastError();
}

}  // namespace mdk
