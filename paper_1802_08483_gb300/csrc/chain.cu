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
//   k_finalize : APPs (eq. L, normalised over D), d logP / d prior and the
//                FP64 reduction of the channel-parameter gradient
//                (k_grad_reduce adds the chunks of a frame in order).
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
constexpr int kChainThreads = 128;
constexpr int kStages = 2;
constexpr uint32_t kWaitLimit = 1u << 26;

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += red[w];  // every thread, same order: same result
    return s;
}

// Two sums at once (normaliser and first moment).
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red) {
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
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < nw; ++w) { sa += red[w]; sb += red[32 + w]; }
    a = sa;
    b = sb;
}

// Tilt controller (see k_chain).
constexpr double kTiltGainMin = 0.02;  // long-run smoothing of the entropy-rate estimate
constexpr double kTiltStepMax = 0.02;  // largest change of the tilt between two rows
constexpr double kTiltMin = 0.2, kTiltMax = 1.6;
constexpr int kTiltEvery = 4;    // steps between tilt updates once settled
constexpr int kTiltSettle = 64;  // updates every step for the first steps

// Geometry of chunk k of the step that consumes W_i.
struct ChunkGeom {
    int d0, d1;     // owned states (alpha: destinations, beta: sources)
    int r0, r1;     // W rows staged
    int shift;      // floats between the aligned copy start and row r0
    uint32_t bytes; // copy size
    const float *src;
};

__device__ __forceinline__ ChunkGeom chunk_geom(const FrameDev &f, int dir, int i, int k) {
    ChunkGeom g;
    const int CD = f.chainCD, M = f.M;
    g.d0 = k * CD;
    g.d1 = min(M, g.d0 + CD);
    if (dir == 0) {  // destination s gets sources s - nI .. s + n
        g.r0 = max(0, g.d0 - f.n * f.I);
        g.r1 = min(M, g.d1 + f.n);
    } else {
        g.r0 = g.d0;
        g.r1 = g.d1;
    }
    const long long o0 = (long long)i * f.wblk + (long long)g.r0 * f.MNS;
    const long long o1 = (long long)i * f.wblk + (long long)g.r1 * f.MNS;
    const long long a0 = o0 & ~3ll;
    const long long a1 = (o1 + 3) & ~3ll;
    g.shift = (int)(o0 - a0);
    g.bytes = (uint32_t)((a1 - a0) * 4);
    if (g.bytes == 0) g.bytes = 16;
    g.src = f.W + a0;
    return g;
}

// Exponential tilt.  The forward metric alpha_i(m) is the joint probability of
// a received prefix of L = n i + m bits, so a row falls off roughly like
// 2^{-h L} (h: entropy rate of the received bits) on top of the drift
// posterior; the backward metric rises the same way.  Far apart in FP32, the
// entries that carry the posterior would underflow.  The chains therefore store
//   alpha^_i(m) = alpha_i(m) 2^{theta_i L} / Z_i,   beta^_i(m) = beta_i(m) 2^{-theta'_i L} / Y_i
// with tilts theta driven toward h by the normalisers: with a tilt theta a
// step's normaliser is about 2^{(theta - h) n}, so theta_{i+1} = theta_i -
// g log2(c_i) / n (g = 1/(steps+1), floored at kTiltGainMin); after the first
// kTiltSettle steps it is updated every kTiltEvery steps from the mean log2 c of
// the steps since.  The producers
// already weight every received bit by 2 (theta = 1), so a step multiplies the
// transition sums by 2^{(theta - 1) j} (j = received length) and pre-scales
// the source row by 2^{(theta_{i+1} - theta_i)(m - mean)}; Z_i and the tilts
// are kept exactly in FP64, and log P(Y) = log alpha^_N(rho - tau) + log Z_N
// - theta_N rho log 2.  The APP producer applies the matching exact factor.
__global__ void __launch_bounds__(kChainThreads) k_chain(const FrameDev *__restrict__ frames,
                                                         const Work *__restrict__ work) {
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    const int dir = wk.tile & 1;  // 0 = forward (alpha), 1 = backward (beta); bit 1: replay
    const int M = f.M, Mp = f.Mp, MNS = f.MNS, MN = f.MN, n = f.n, N = f.N, xmax = f.xmax;
    const long long rho = f.rho;
    const int CD = f.chainCD;
    const int nck = (M + CD - 1) / CD;
    const int i0 = f.seg_i0, i1 = f.seg_i1;  // symbols of this launch (segment)
    const long long total = (long long)(i1 - i0) * nck;
    const int send = (int)(rho - (long long)n * N) + xmax;  // state of the end drift
    const bool segm = (f.chain_flags & CH_SEGMENTED) != 0;
    const bool replay = dir == 0 && (wk.tile & 2) != 0;
    // first launch of this direction: the frame boundary; otherwise the row carried over
    const bool fresh = dir == 0 ? (i0 == 0) : (i1 == N);

    __shared__ uint64_t bar[kStages];
    __shared__ double red[64];
    __shared__ int s_fail;
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
        for (int st = 0; st < kStages; ++st) mbar_init(&bar[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    {
        float *row0 = (dir == 0) ? f.alpha + (size_t)i0 * Mp : f.beta + (size_t)i1 * Mp;
        for (int s = threadIdx.x; s < Mp; s += blockDim.x) row0[s] = cur[s];
    }
    auto step_symbol = [&](long long g) -> int {
        const int st = (int)(g / nck);
        return dir == 0 ? i0 + st : i1 - 1 - st;
    };
    // Self-check of every copy: source inside this frame's W, destination inside
    // its stage, 16-byte alignment and size.  A violation records ST_ARG in the
    // frame status and completes the stage's phase with a plain arrive instead.
    const float *wlo = f.W + (size_t)i0 * f.wblk;
    const float *whi = f.W + (size_t)i1 * f.wblk + 16;
    auto issue = [&](long long g) {
        const int i = step_symbol(g);
        const int k = (int)(g % nck);
        const ChunkGeom cg = chunk_geom(f, dir, i, k);
        uint64_t *b = &bar[g % kStages];
        float *dst = stage0 + (size_t)(g % kStages) * stageFloats;
        const bool ok = cg.src >= wlo && cg.src + cg.bytes / 4 <= whi &&
                        cg.bytes % 16 == 0 && cg.bytes / 4 <= stageFloats &&
                        ((uintptr_t)cg.src & 15) == 0 && ((uintptr_t)dst & 15) == 0;
        if (ok) {
            mbar_expect_tx(b, cg.bytes);
            bulk_g2s(dst, cg.src, cg.bytes, b);
        } else {
            atomicMax(f.status, ST_ARG);
            mbar_arrive(b);
        }
    };
    if (threadIdx.x == 0)
        for (long long g = 0; g < kStages && g < total; ++g) issue(g);

    __shared__ double s_th[3];  // tilt of the current row, of the row being built, row mean
    __shared__ float vfac[kMaxMN];
    double logZ = 0.0;       // thread 0: log Z_i (forward) in nats
    double theta = 1.0;      // thread 0: tilt of the current row
    double mean = (dir == 0) ? 0.0 : (double)(send - xmax);  // thread 0: mean drift of it
    double lc_prev = 0.0;    // thread 0: sum of log2 c since the last tilt update
    int lc_cnt = 0;          // thread 0: number of steps in lc_prev
    long long steps = 0;     // every thread: steps taken in this direction so far
    if (!fresh && segm) {
        const ChainState &cs = f.cst[dir];
        steps = cs.steps;
        if (threadIdx.x == 0) {
            theta = cs.theta;
            mean = cs.mean;
            logZ = cs.logZ;
            lc_prev = cs.lc_sum;
            lc_cnt = cs.lc_cnt;
        }
    }
    if (replay) steps = i0;
    if (threadIdx.x == 0 && fresh && !replay) {
        if (dir == 0) { f.thf[0] = 1.0; f.mcf[0] = 0.0; }
        else f.thb[N] = 1.0;
    }
    double part = 0.0, partm = 0.0;  // this thread's share of the normaliser and first moment
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
        th_cur = th_new = (float)s_th[0];
        mc = (float)s_th[2];
        for (int j = threadIdx.x; j < MN; j += blockDim.x) vfac[j] = exp2f((th_cur - 1.f) * (float)j);
        __syncthreads();
    }
    bool failed = false;
    long long gfail = 0;
    for (long long g = 0; g < total; ++g) {
        const int i = step_symbol(g);
        const int k = (int)(g % nck);
        const bool update = replay || steps < kTiltSettle || (steps % kTiltEvery) == 0;
        if (k == 0 && update) {
            // start of an update step: choose the tilt of the rows from here on
            // (the recompute sweep replays the tilts recorded by the first sweep)
            if (threadIdx.x == 0 && replay) {
                s_th[0] = f.thf[i];
                s_th[1] = f.thf[i + 1];
                s_th[2] = f.mcf[i];
            } else if (threadIdx.x == 0) {
                double tn = theta;
                if (steps > 0 && lc_cnt > 0) {
                    const double gain =
                        fmin(1.0, fmax(kTiltGainMin, (double)lc_cnt / (double)(steps + 1)));
                    const double d =
                        fmin(kTiltStepMax, fmax(-kTiltStepMax, -gain * (lc_prev / lc_cnt) / n));
                    tn = fmin(kTiltMax, fmax(kTiltMin, theta + d));
                }
                s_th[0] = theta;
                s_th[1] = tn;
                s_th[2] = mean;
                lc_prev = 0.0;
                lc_cnt = 0;
            }
            __syncthreads();
            th_cur = (float)s_th[0];
            th_new = (float)s_th[1];
            mc = (float)s_th[2];
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
        const ChunkGeom cg = chunk_geom(f, dir, i, k);
        const float *buf = stage0 + (size_t)(g % kStages) * stageFloats + cg.shift;
        if (!mbar_wait(&bar[g % kStages], (uint32_t)((g / kStages) & 1), kWaitLimit)) {
            atomicExch(&s_fail, ST_TIMEOUT);
        }
        // valid source rows: window start p = n i + s - xmax inside [0, rho]
        const int vlo = max(0, (int)max(0ll, (long long)xmax - (long long)n * i));
        const long long vhi_l = rho - (long long)n * i + xmax;
        const int vhi = (int)min((long long)M - 1, vhi_l);
        if (dir == 0) {
            const int lo = max(cg.r0, vlo), hi = min(cg.r1 - 1, vhi);
            for (int s = cg.d0 + threadIdx.x; s < cg.d1; s += blockDim.x) {
                float acc = 0.f;
                const int jlo = max(0, s + n - hi), jhi = min(MN - 1, s + n - lo);
                for (int j = jlo; j <= jhi; ++j) {
                    const int src = s - j + n;
                    acc = fmaf(cur[src], buf[(size_t)(src - cg.r0) * MNS + j] * vfac[j], acc);
                }
                nxt[s] = acc;
                part += (double)acc;
                partm += (double)acc * (double)(s - xmax);
            }
        } else {
            const float dth = th_cur - th_new;  // post-scale 2^{(theta'_{i+1} - theta'_i)(m - mean)}
            for (int s = cg.d0 + threadIdx.x; s < cg.d1; s += blockDim.x) {
                float acc = 0.f;
                if (s >= vlo && s <= vhi) {
                    const int jlo = max(0, n - s), jhi = min(MN - 1, M - 1 - s + n);
                    const float *w = buf + (size_t)(s - cg.r0) * MNS;
                    for (int j = jlo; j <= jhi; ++j)
                        acc = fmaf(w[j] * vfac[j], cur[s + j - n], acc);
                    if (dth != 0.f) acc *= exp2f(dth * ((float)(s - xmax) - mc));
                }
                nxt[s] = acc;
                part += (double)acc;
                partm += (double)acc * (double)(s - xmax);
            }
        }
        __syncthreads();  // stage consumed by everyone
        if (threadIdx.x == 0 && g + kStages < total) issue(g + kStages);
        if (k == nck - 1) {
            // end of a step: normalise, keep the FP64 record
            double c = part, cm = partm;
            block_sum2(c, cm, red);
            part = 0.0;
            partm = 0.0;
            if (!(c > 0.0) || !isfinite(c)) {
                if (threadIdx.x == 0) atomicCAS(&s_fail, 0, ST_ZERO);
            }
            __syncthreads();
            if (s_fail) { failed = true; gfail = g; break; }
            const float inv = (float)(1.0 / c);
            if (threadIdx.x == 0) {
                const double dth = (double)th_new - (double)th_cur;
                if (dir == 0 && !replay) {
                    logZ += log(c) + dth * ((double)n * i + (double)mc) * 0.6931471805599453;
                    f.thf[i + 1] = (double)th_new;
                    f.mcf[i + 1] = cm / c;
                } else if (dir == 1) {
                    f.thb[i] = (double)th_new;
                }
                theta = (double)th_new;
                mean = cm / c;
                lc_prev += log2(c);
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
    }
    if (failed) {
        // Copies already issued (chunks g+1 .. g+kStages) must land before the
        // CTA's shared memory is released: wait for them, again with a bound.
        if (threadIdx.x == 0) {
            for (long long h = gfail + 1; h <= gfail + kStages && h < total; ++h)
                mbar_wait(&bar[h % kStages], (uint32_t)((h / kStages) & 1), kWaitLimit);
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
            cs.logZ = logZ;
            cs.lc_sum = lc_prev;
            cs.lc_cnt = lc_cnt;
            cs.steps = steps;
        }
    }
    if (dir == 0 && !replay && i1 == N && threadIdx.x == 0) {
        const float aN = cur[send];
        if (!(aN > 0.f)) {
            atomicMax(f.status, ST_ZERO);
        } else {
            *f.loglik = log((double)aN) + logZ - theta * (double)rho * 0.6931471805599453;
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
    const int q = f.q, n = f.n, N = f.N, xmax = f.xmax;
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
        const int tlo = (int)(plo / P2), thi = (int)(phi / P2);
        // lane l holds the Lp row offset of super-tile tlo + l for this symbol
        long long myrow = 0;
        if (tlo + lane <= thi) {
            int ilo, ihi;
            super_symbols(f, tlo + lane, ilo, ihi);
            myrow = (long long)(tlo + lane) * f.S2 + (i - ilo);
        }
        double z = 0.0;
        // pass 1: unnormalised sums into app, and z = sum_D prior(D) L^u(D)
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
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        if (!(z > 0.0)) { bad = true; continue; }
        const double iz = 1.0 / z;
        // pass 2: each lane rescales the entries it wrote
        for (int D = lane; D < q; D += 32) {
            const size_t e = (size_t)i * q + D;
            const double lu = (double)f.app[e];
            f.app[e] = (float)((double)f.priors[e] * lu * iz);
            if (f.dpriors) f.dpriors[e] = (float)(lu * iz);
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
// Launch wrappers (host).
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
    return 4 * (2 * (size_t)f.Mp + kStages * stageFloats);
}

cudaError_t launch_chain(const FrameDev *frames, const Work *work, int nwork, size_t smem,
                         cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    // Raise the opt-in limit once to the device maximum: graphs hold chain launches
    // of several waves with different sizes, and every one must stay valid.
    static int max_dyn = -1;
    if (max_dyn < 0) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k_chain);
        if (e != cudaSuccess) return e;
        int dev = 0, optin = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        const int lim = optin - (int)fa.sharedSizeBytes;
        e = cudaFuncSetAttribute(k_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e != cudaSuccess) return e;
        max_dyn = lim;
    }
    if ((long long)smem > max_dyn) return cudaErrorInvalidValue;
    k_chain<<<nwork, kChainThreads, smem, st>>>(frames, work);
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
