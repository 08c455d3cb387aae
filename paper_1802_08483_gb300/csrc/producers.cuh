// Producer kernels: the parallel parts of the decoder, one CTA per
// (frame, tile of P received positions).
//
//   k_fwd  : receiver metric R[p][D][j] for the tile's positions (lattice,
//            eqs. F / F_lastrow) into shared memory, then the prior-weighted
//            transition sums  W_i(s', j) = sum_D prior_i(D) R[n i + m'][D][j]
//            (eq. gamma summed over D) for every symbol i whose window starts
//            in the tile.  W feeds the forward and backward recursions.
//   k_bwd  : recomputes R for the tile and forms, for each touched symbol i,
//            sum_{m', j} alpha_i(m') R[p][D][j] beta_{i+1}(m'+j-n)  (eqs. L,
//            sigma without the prior) as a partial sum per tile; in gradient
//            mode also the same sums with dR/dw, dR/dPd, dR/d(Pt Ps).
//   k_rmetric : step (1) alone, R dumped to global memory.
//
// Included by one translation unit per insertion cap; NB == 0 selects the
// run-time (n, I) lattice.
#pragma once

#include "mapdec_dev.cuh"

namespace mdk {

template <int NB, int IB, int MODE>
__device__ __forceinline__ void lattice_any(const FrameDev &f, uint32_t x, uint64_t y,
                                            float *Fout, float *Tout) {
    if constexpr (NB == 0) {
        lattice_runtime<MODE>(f.n, f.I, x, y, f.wpow, f.wder, f.Pd, f.qsame, f.qdiff, Fout,
                              Tout);
    } else {
        constexpr int MN = NB * (IB + 1) + 1;
        float F[MN], T[MN];
        lattice_unrolled<NB, IB, MODE>(x, y, f.wpow, f.wder, f.Pd, f.qsame, f.qdiff, F, T);
#pragma unroll
        for (int j = 0; j < MN; ++j) {
            Fout[j] = F[j];
            if (MODE) Tout[j] = T[j];
        }
    }
}

// Evaluate lattice (p, D); out[j] for j < MN, zero where p + j > rho.
// MODE 0 -> R; MODE k > 0 -> the k-th tangent.
template <int NB, int IB, int MODE>
__device__ __forceinline__ void eval_metric(const FrameDev &f, long long p, int D, float *out) {
    const int MN = (NB == 0) ? f.MN : NB * (IB + 1) + 1;
    float F[kMaxMN], T[kMaxMN];
    const uint64_t y = rx_window(f.rxbits, p);
    const uint32_t x = __ldg(f.cw + D);
    lattice_any<NB, IB, MODE>(f, x, y, F, T);
    const long long lim = f.rho - p;
#pragma unroll
    for (int j = 0; j < ((NB == 0) ? kMaxMN : NB * (IB + 1) + 1); ++j) {
        if (j < MN) {
            const float v = MODE ? T[j] : F[j];
            out[j] = (j <= lim) ? v : 0.f;
        }
    }
}

// ---------------------------------------------------------------------------
// Forward producer.
// smem: Rs[q][RS]  (RS = roundup4(P*MN); column c = pl*MN + j)
//       Pr[q][S4]  (priors of the touched symbols, transposed)
// ---------------------------------------------------------------------------
template <int NB, int IB>
__device__ __forceinline__ void fwd_body(const FrameDev *__restrict__ frames,
                                         const Work *__restrict__ work) {
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    const int n = (NB == 0) ? f.n : NB;
    const int MN = (NB == 0) ? f.MN : NB * (IB + 1) + 1;
    const int q = f.q, P = f.Pf, M = f.M, xmax = f.xmax;
    const long long rho = f.rho;
    const long long p0 = (long long)wk.tile * P;
    int ilo, ihi;
    tile_symbols(f, wk.tile, ilo, ihi);
    const int S = ihi - ilo + 1;
    if (S <= 0) return;
    const int S4 = (S + 3) & ~3;
    const int NC = P * MN;
    const int RS = (NC + 3) & ~3;

    extern __shared__ float4 smem4[];
    float *Rs = reinterpret_cast<float *>(smem4);
    float *Pr = Rs + (size_t)q * RS;

    // (A) receiver metrics of the tile; a warp covers consecutive p for one D.
    for (int idx = threadIdx.x; idx < P * q; idx += blockDim.x) {
        const int D = idx / P, pl = idx - D * P;
        const long long p = p0 + pl;
        float *dst = Rs + (size_t)D * RS + pl * MN;
        if (p <= rho) {
            float v[kMaxMN];
            eval_metric<NB, IB, 0>(f, p, D, v);
            for (int j = 0; j < MN; ++j) dst[j] = v[j];
        } else {
            for (int j = 0; j < MN; ++j) dst[j] = 0.f;
        }
    }
    for (int idx = threadIdx.x; idx < q * (RS - NC); idx += blockDim.x) {
        const int D = idx / (RS - NC), c = NC + idx % (RS - NC);
        Rs[(size_t)D * RS + c] = 0.f;
    }
    __syncthreads();
    if (f.Rg) {
        // keep R for the APP producer: rows pl*MN + j, columns D (zero-padded to DS)
        const int DS = (q + 3) & ~3;
        float *dst = f.Rg + (size_t)wk.tile * NC * DS;
        for (int idx = threadIdx.x; idx < NC * DS; idx += blockDim.x) {
            const int row = idx / DS, D = idx - row * DS;
            dst[idx] = D < q ? Rs[(size_t)D * RS + row] : 0.f;
        }
    }
    // (B) priors of the touched symbols, transposed to [D][il]
    for (int idx = threadIdx.x; idx < S4 * q; idx += blockDim.x) {
        const int il = idx / q, D = idx - il * q;
        Pr[(size_t)D * S4 + il] = (il < S) ? __ldg(f.priors + (size_t)(ilo + il) * q + D) : 0.f;
    }
    __syncthreads();

    // (C) W tile = Pr^T (S x q) * Rs (q x NC), 4x4 register micro-tiles;
    // only entries with start drift inside the limits are stored.
    const int NRG = S4 / 4, NCG = RS / 4;
    for (int idx = threadIdx.x; idx < NRG * NCG; idx += blockDim.x) {
        const int rg = idx / NCG, cg = idx - rg * NCG;
        const int il0 = rg * 4, c0 = cg * 4;
        // band test on the micro-tile corners
        const long long pA = p0 + c0 / MN, pB = p0 + min(c0 + 3, NC - 1) / MN;
        const long long sMin = pA - (long long)n * (ilo + il0 + 3) + xmax;
        const long long sMax = pB - (long long)n * (ilo + il0) + xmax;
        if (sMax < 0 || sMin >= M || c0 >= NC) continue;
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[r][t] = 0.f;
        for (int D = 0; D < q; ++D) {
            const float4 a = *reinterpret_cast<const float4 *>(Pr + (size_t)D * S4 + il0);
            const float4 b = *reinterpret_cast<const float4 *>(Rs + (size_t)D * RS + c0);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int t = 0; t < 4; ++t) acc[r][t] = fmaf(av[r], bv[t], acc[r][t]);
        }
        // rows of W are contiguous in (s', j) when MNS == MN: the 4 columns of a
        // micro-tile land on consecutive floats unless the band clips them
        const long long pBlast = p0 + (c0 + 3 < NC ? c0 + 3 : NC - 1) / MN;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int il = il0 + r;
            if (il >= S) break;
            const long long i = ilo + il;
            float *Wi = f.W + (size_t)i * f.wblk;
            const long long sA = pA - (long long)n * i + xmax;
            const long long sB = pBlast - (long long)n * i + xmax;
            if (f.MNS == MN && c0 + 3 < NC && sA >= 0 && sB < M && pBlast <= rho) {
                float *dst = Wi + (p0 - (long long)n * i + xmax) * MN + c0;
#pragma unroll
                for (int t = 0; t < 4; ++t) dst[t] = acc[r][t];
                continue;
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int c = c0 + t;
                if (c >= NC) break;
                const int pl = c / MN, j = c - pl * MN;
                const long long p = p0 + pl;
                const long long s = p - (long long)n * i + xmax;
                if (s >= 0 && s < M && p <= rho) Wi[s * f.MNS + j] = acc[r][t];
            }
        }
    }
}

// Two register budgets: the compiler's own (I <= 2 classes fit two CTAs per SM
// with it) and at most 128 registers (I >= 3, whose longer lattice rows would
// otherwise hold one CTA per SM).
template <int NB, int IB>
__global__ void __launch_bounds__(kThreads) k_fwd(const FrameDev *__restrict__ frames,
                                                  const Work *__restrict__ work) {
    fwd_body<NB, IB>(frames, work);
}
template <int NB, int IB>
__global__ void __launch_bounds__(kThreads, 2) k_fwd_occ2(const FrameDev *__restrict__ frames,
                                                          const Work *__restrict__ work) {
    fwd_body<NB, IB>(frames, work);
}

// ---------------------------------------------------------------------------
// alpha and beta windows of an APP-producer sub-tile (positions p0 .. p0+P-1,
// symbols ilo .. ilo+S-1, row stride S4 >= S), with the exact factor that
// undoes the chains' tilts (k_chain):
//   sigma ~ alpha^_i(m') beta^_{i+1}(m) 2^{(theta'_{i+1} - theta_i)(m' - mean_i)}
//           2^{(theta'_{i+1} - 1) j} prior R~
// up to a constant per symbol.  The per-j factor 2^{phi j}, phi =
// theta'_{i+1} - 1, splits exactly as 2^{phi (pl + j)} 2^{-phi pl}: folded
// into the beta window (index pl + j) and the alpha window (index pl).
// With m' = p0 + pl - n i the alpha-side exponent is e0_i + g_i pl,
// e0_i = (theta'_{i+1} - theta_i)(p0 - n i - mean_i) (split into integer and
// fraction), g_i = theta'_{i+1} - theta_i - phi; the factor is applied as
// alpha 2^frac scaled by 2^int (exact), clamped below overflow.  The tilts
// and means are FP32 values, so e0_i is formed exactly enough in FP32 pairs
// (error-free sum and product): its integer part exactly, its fraction to a
// few FP32 ulps.
// Windows: Aw[pl][il] = alpha_i(state of p0 + pl), Bw[k][il] =
// beta_{i+1}(state of p0 - n + k), k < BW = P + MN - 1, zero outside the
// limits or past rho.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void window_constants(const FrameDev &f, long long p0, int n, int ilo,
                                                 int S, int S4, int *symE, float *symF,
                                                 float *symG, float *symPhi) {
    for (int il = threadIdx.x; il < S4; il += blockDim.x) {
        int ei = 0;
        float ef = 0.f, g = 0.f, phi = 0.f;
        if (il < S) {
            const long long i = ilo + il;
            const float tb = (float)f.thb[i + 1], tf = (float)f.thf[i];
            const float mu = (float)f.mcf[i];
            // dth = tb - tf and x = (p0 - n i) - mu as unevaluated sums hi + lo
            float dh, dl, xh, xl;
            two_sum(tb, -tf, dh, dl);
            two_sum((float)(p0 - (long long)n * i), -mu, xh, xl);
            // e0 = dth x = ph + pl + (dh xl + dl xh) (dl xl is far below FP32 ulp)
            const float ph0 = dh * xh;
            const float pl0 = fmaf(dh, xh, -ph0);
            const float r = rintf(ph0);
            ei = (int)fmaxf(-100000.f, fminf(100000.f, r));
            ef = ((ph0 - r) + pl0) + fmaf(dh, xl, dl * xh);
            phi = tb - 1.f;
            g = (dh - phi) + dl;
        }
        symE[il] = ei;
        symF[il] = ef;
        symG[il] = g;
        symPhi[il] = phi;
    }
}

// Raw rows fetched row by row (coalesced) by 4-byte asynchronous copies; the
// caller waits for them (cp_async_wait_all) and a CTA barrier before use.
// One symbol per warp, positions across the lanes (no divisions).
__device__ __forceinline__ void window_fetch(const FrameDev &f, long long p0, int n, int ilo,
                                             int S, int S4, int P, int BW, float *Aw,
                                             float *Bw) {
    const int M = f.M, xmax = f.xmax;
    const long long rho = f.rho;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, NW = blockDim.x >> 5;
    for (int il = warp; il < S4; il += NW) {
        const long long i = ilo + il;
        const long long sa = p0 - (long long)n * i + xmax;  // state of position p0
        const float *arow = f.alpha + (size_t)i * f.Mp;
        const float *brow = f.beta + (size_t)(i + 1) * f.Mp;
        for (int pl = lane; pl < P; pl += 32) {
            const long long s = sa + pl;
            float *dst = Aw + pl * S4 + il;
            if (il < S && s >= 0 && s < M && p0 + pl <= rho) cp_async4(dst, arow + s);
            else *dst = 0.f;
        }
        for (int k = lane; k < BW; k += 32) {
            const long long s = sa - n + k;
            float *dst = Bw + k * S4 + il;
            if (il < S && s >= 0 && s < M) cp_async4(dst, brow + s);
            else *dst = 0.f;
        }
    }
}

// The tilt factors applied in place to the landed windows.
__device__ __forceinline__ void window_tilt(int S, int S4, int P, int BW, float *Aw, float *Bw,
                                            const int *symE, const float *symF,
                                            const float *symG, const float *symPhi) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, NW = blockDim.x >> 5;
    for (int il = warp; il < S; il += NW) {
        const float g = symG[il], fr = symF[il], phi = symPhi[il];
        const int e0 = symE[il];
        for (int pl = lane; pl < P; pl += 32) {
            float *ap = Aw + pl * S4 + il;
            const float a = *ap;
            if (a > 0.f) {
                const float e = fmaf(g, (float)pl, fr);
                const float k = rintf(e);
                const int ex = min(max(e0 + (int)k, -300), 300);
                // 2^ex as two exact powers of two within the FP32 exponent range
                const int e1 = min(max(ex, -126), 127);
                const int e2 = min(max(ex - e1, -126), 127);
                const float v = a * exp2f(e - k);
                *ap = fminf(v * pow2i(e1) * pow2i(e2), 3.0e38f);
            }
        }
        for (int k = lane; k < BW; k += 32) {
            float *bp = Bw + k * S4 + il;
            const float b = *bp;
            if (b != 0.f) *bp = b * exp2f(phi * (float)k);
        }
    }
}

// ---------------------------------------------------------------------------
// Backward producer (APP partial sums, optional tangents).  One CTA owns a
// super-tile of nsub sub-tiles of P positions and accumulates, in shared
// memory, for every symbol i it touches:
//   Lacc[i][D] = sum_{p in super-tile, j} alpha_i(s') R[p][D][j] beta_{i+1}(s'+j-n)
//   Gacc[i][t] = sum_D prior_i(D) (the same sum with the t-th tangent of R)
// Per sub-tile the contraction is evaluated as
//   C[i][c] = sum_pl Aw[pl][i] * ( sum_j Bw[pl+j][i] * Rt[pl*MN+j][c] ),
// i.e. the dense GEMM C(S x NR*DS) = AB(S x P*MN) * Rt(P*MN x NR*DS) with the
// A operand AB = alpha (x) beta factored, so it is never materialised.
// smem: Rt[K][CW]  (K = P*MN, CW = NR*DS, DS = roundup4(q); column t*DS + D)
//       Aw[P][S4], Bw[BW][S4] (BW = P + MN - 1), both carrying the tilt factors
//       symbol constants (3 x S4), Lacc[S2][q], Gacc[S2][3], Ct[3][S4][DS] (gradient)
// ---------------------------------------------------------------------------
template <int NB, int IB, bool GRAD>
__global__ void __launch_bounds__(kThreads, (GRAD && (NB == 0 || NB > 10)) ? 1 : 2) k_bwd(const FrameDev *__restrict__ frames,
                                                     const Work *__restrict__ work) {
    constexpr int NR = GRAD ? 4 : 1;
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    const int n = (NB == 0) ? f.n : NB;
    const int MN = (NB == 0) ? f.MN : NB * (IB + 1) + 1;
    const int q = f.q, P = f.P;
    const long long rho = f.rho;
    int ilo2, ihi2;
    super_symbols(f, wk.tile, ilo2, ihi2);
    const int S2 = ihi2 - ilo2 + 1;
    if (S2 <= 0) return;
    const int DS = (q + 3) & ~3;
    const int CW = NR * DS;
    const int K = P * MN;
    const int BW = P + MN - 1;
    const int Smax4 = (f.S + 3) & ~3;

    extern __shared__ float4 smem4[];
    float *Rt = reinterpret_cast<float *>(smem4);
    float *Aw = Rt + (size_t)K * CW;
    float *Bw = Aw + (size_t)P * Smax4;
    int *symE = reinterpret_cast<int *>(Bw + (size_t)BW * Smax4);  // integer part of the alpha-side exponent
    float *symF = reinterpret_cast<float *>(symE + Smax4);      // its fraction
    float *symG = symF + Smax4;                                 // its slope in pl
    float *symPhi = symG + Smax4;                               // theta'_{i+1} - 1
    float *Lacc = symPhi + Smax4;
    float *Gacc = Lacc + (((size_t)f.S2 * q + 3) & ~(size_t)3);
    float *Ct = Gacc + (((size_t)f.S2 * 3 + 3) & ~(size_t)3);

    for (int idx = threadIdx.x; idx < S2 * q; idx += blockDim.x) Lacc[idx] = 0.f;
    if (GRAD)
        for (int idx = threadIdx.x; idx < S2 * 3; idx += blockDim.x) Gacc[idx] = 0.f;

    for (int sub = 0; sub < f.nsub; ++sub) {
        const long long p0 = ((long long)wk.tile * f.nsub + sub) * P;
        if (p0 > rho) break;
        int ilo, ihi;
        range_symbols(f, p0, p0 + P - 1, ilo, ihi);
        const int S = ihi - ilo + 1;
        if (S <= 0) continue;
        const int S4 = (S + 3) & ~3;
        const int off = ilo - ilo2;  // row of symbol ilo in the accumulators

        // (B) alpha and beta windows of the sub-tile's symbols (see
        // window_constants / window_fetch); the raw rows land while the
        // lattices below run.
        window_constants(f, p0, n, ilo, S, S4, symE, symF, symG, symPhi);
        window_fetch(f, p0, n, ilo, S, S4, P, BW, Aw, Bw);

        // (A) receiver metrics (and tangents); lanes cover consecutive D for one p.
        // Decode mode with stored metrics: copy the tile's block instead.
        if (!GRAD && f.Rg) {
            const float4 *src = reinterpret_cast<const float4 *>(
                f.Rg + ((size_t)wk.tile * f.nsub + sub) * (size_t)K * DS);
            float4 *dst = reinterpret_cast<float4 *>(Rt);
            for (int idx = threadIdx.x; idx < K * DS / 4; idx += blockDim.x) dst[idx] = __ldg(src + idx);
        }
        for (int idx = threadIdx.x; idx < ((!GRAD && f.Rg) ? 0 : P * q); idx += blockDim.x) {
            const int pl = idx / q, D = idx - pl * q;
            const long long p = p0 + pl;
#pragma unroll
            for (int th = 0; th < NR; ++th) {
                float v[kMaxMN];
                if (p <= rho) {
                    if (th == 0) eval_metric<NB, IB, 0>(f, p, D, v);
                    if (GRAD && th == 1) eval_metric<NB, IB, 1>(f, p, D, v);
                    if (GRAD && th == 2) eval_metric<NB, IB, 2>(f, p, D, v);
                    if (GRAD && th == 3) eval_metric<NB, IB, 3>(f, p, D, v);
                } else {
                    for (int j = 0; j < MN; ++j) v[j] = 0.f;
                }
                float *dst = Rt + (size_t)pl * MN * CW + th * DS + D;
                for (int j = 0; j < MN; ++j) dst[(size_t)j * CW] = v[j];
            }
        }
        if (DS > q && (GRAD || !f.Rg)) {
            for (int idx = threadIdx.x; idx < K * NR * (DS - q); idx += blockDim.x) {
                const int row = idx / (NR * (DS - q)), r2 = idx - row * (NR * (DS - q));
                const int th = r2 / (DS - q), col = q + r2 % (DS - q);
                Rt[(size_t)row * CW + th * DS + col] = 0.f;
            }
        }
        // (B) the windows' raw alpha/beta values have landed: apply the tilt
        // factors in place.
        cp_async_wait_all();
        __syncthreads();
        window_tilt(S, S4, P, BW, Aw, Bw, symE, symF, symG, symPhi);
        __syncthreads();

        // (C) register micro-tiles of 4 symbols x 4 columns.  With fewer
        // micro-tiles than threads, KS adjacent lanes share one micro-tile and
        // split the positions; their partial sums combine by shuffles, in a
        // fixed order.
        const int NRG = S4 / 4, NCG = CW / 4;
        const int NMT = NRG * NCG;
        int KS = 1;
        while (KS < 32 && KS * 2 <= P && NMT * KS * 2 <= (int)blockDim.x) KS *= 2;
        const int units = NMT * KS;
        const float4 *Aw4 = reinterpret_cast<const float4 *>(Aw);
        const float4 *Bw4 = reinterpret_cast<const float4 *>(Bw);
        const float4 *Rt4 = reinterpret_cast<const float4 *>(Rt);
        const int sr = S4 / 4, cr = CW / 4;
        for (int u0 = 0; u0 < units; u0 += blockDim.x) {
            const int u = u0 + (int)threadIdx.x;
            const bool active = u < units;
            const int mt = active ? u / KS : 0;
            const int ks = u & (KS - 1);
            const int rg = mt / NCG, cg = mt - rg * NCG;
            float acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
            if (active) {
                for (int pl = ks; pl < P; pl += KS) {
                    const float4 a = Aw4[pl * sr + rg];
                    if (a.x == 0.f && a.y == 0.f && a.z == 0.f && a.w == 0.f) continue;
                    float t[4][4];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) t[r][c] = 0.f;
                    const float4 *bp = Bw4 + pl * sr + rg;
                    const float4 *rp = Rt4 + (size_t)pl * MN * cr + cg;
#pragma unroll 8
                    for (int j = 0; j < MN; ++j) {
                        const float4 b = bp[j * sr];
                        const float4 rr = rp[j * cr];
                        const float bv[4] = {b.x, b.y, b.z, b.w};
                        const float rv[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int c = 0; c < 4; ++c) t[r][c] = fmaf(bv[r], rv[c], t[r][c]);
                    }
                    const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], t[r][c], acc[r][c]);
                }
            }
            for (int o = 1; o < KS; o <<= 1) {
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], o);
            }
            // (D) owners add into the accumulators / stage tangent sums
            if (active && ks == 0) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int il = rg * 4 + r;
                    if (il >= S) break;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int col = cg * 4 + c;
                        const int th = col / DS, D = col - th * DS;
                        if (D >= q) continue;
                        if (th == 0) Lacc[(size_t)(off + il) * q + D] += acc[r][c];
                        else Ct[((size_t)(th - 1) * Smax4 + il) * DS + D] = acc[r][c];
                    }
                }
            }
        }
        if (GRAD) {
            __syncthreads();
            for (int idx = threadIdx.x; idx < 3 * S; idx += blockDim.x) {
                const int tt = idx / S, il = idx - tt * S;
                const float *pr = f.priors + (size_t)(ilo + il) * q;
                const float *ct = Ct + ((size_t)tt * Smax4 + il) * DS;
                float s = 0.f;
                for (int D = 0; D < q; ++D) s = fmaf(__ldg(pr + D), ct[D], s);
                Gacc[(off + il) * 3 + tt] += s;
            }
        }
        __syncthreads();
    }
    const size_t row0 = (size_t)wk.tile * f.S2;
    for (int idx = threadIdx.x; idx < S2 * q; idx += blockDim.x)
        f.Lp[row0 * q + idx] = Lacc[idx];
    if (GRAD)
        for (int idx = threadIdx.x; idx < S2 * 3; idx += blockDim.x)
            f.Gp[row0 * 3 + idx] = Gacc[idx];
}

// Step (1) alone: one thread per (p, D).
template <int NB, int IB>
__global__ void __launch_bounds__(kThreads) k_rmetric(const FrameDev *__restrict__ frames) {
    const FrameDev &f = frames[0];
    const int MN = (NB == 0) ? f.MN : NB * (IB + 1) + 1;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (f.rho + 1) * f.q;
    if (idx >= total) return;
    const long long p = idx / f.q;
    const int D = (int)(idx - p * f.q);
    float v[kMaxMN];
    eval_metric<NB, IB, 0>(f, p, D, v);
    float *dst = f.Rout + idx * MN;
    // undo the received-bit weight kappa^j (a power of two: exact)
    const int lk = (int)lrint(f.logk / 0.6931471805599453);
    for (int j = 0; j < MN; ++j) dst[j] = ldexpf(v[j], -lk * j);
}

}  // namespace mdk
