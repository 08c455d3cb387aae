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
__global__ void __launch_bounds__(kThreads) k_fwd(const FrameDev *__restrict__ frames,
                                                  const Work *__restrict__ work) {
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    const int n = (NB == 0) ? f.n : NB;
    const int MN = (NB == 0) ? f.MN : NB * (IB + 1) + 1;
    const int q = f.q, P = f.P, M = f.M, xmax = f.xmax;
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

// ---------------------------------------------------------------------------
// Backward producer (APP partial sums, optional tangents).  One CTA owns a
// super-tile of nsub sub-tiles of P positions and accumulates, in shared
// memory, for every symbol i it touches:
//   Lacc[i][D] = sum_{p in super-tile, j} alpha_i(s') R[p][D][j] beta_{i+1}(s'+j-n)
//   Gacc[i][t] = sum_D prior_i(D) (the same sum with the t-th tangent of R)
// Per sub-tile this is a GEMM  C (S x NR*DS) = AB (S x K) * Rt (K x NR*DS),
// K = P*MN, whose A operand AB[c][il] = alpha*beta is built in chunks.
// smem: Rt[K][CW]  (CW = NR*DS, DS = roundup4(q); column t*DS + D)
//       Aw[S][P], Bw[S][BW] (BW = P + MN - 1), both carrying the tilt factors
//       AB[kKC][S4] / reduction scratch
//       Lacc[S2][q], Gacc[S2][3], Ct[3][S4][DS] (gradient mode)
// ---------------------------------------------------------------------------
constexpr int kKC = 32;  // K chunk

template <int NB, int IB, bool GRAD>
__global__ void __launch_bounds__(kThreads) k_bwd(const FrameDev *__restrict__ frames,
                                                  const Work *__restrict__ work) {
    constexpr int NR = GRAD ? 4 : 1;
    constexpr int MT = 4;  // micro-tiles per thread
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    const int n = (NB == 0) ? f.n : NB;
    const int MN = (NB == 0) ? f.MN : NB * (IB + 1) + 1;
    const int q = f.q, P = f.P, M = f.M, xmax = f.xmax;
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
    float *Bw = Aw + (((size_t)f.S * P + 3) & ~(size_t)3);
    float *AB = Bw + (((size_t)f.S * BW + 3) & ~(size_t)3);
    size_t abn = (size_t)kKC * Smax4;
    if (abn < (size_t)kThreads * 16) abn = (size_t)kThreads * 16;
    float *Lacc = AB + abn;
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

        // (A) receiver metrics (and tangents); lanes cover consecutive D for one p.
        for (int idx = threadIdx.x; idx < P * q; idx += blockDim.x) {
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
        if (DS > q) {
            for (int idx = threadIdx.x; idx < K * NR * (DS - q); idx += blockDim.x) {
                const int row = idx / (NR * (DS - q)), r2 = idx - row * (NR * (DS - q));
                const int th = r2 / (DS - q), col = q + r2 % (DS - q);
                Rt[(size_t)row * CW + th * DS + col] = 0.f;
            }
        }
        // (B) alpha and beta windows of the sub-tile's symbols, with the exact
        // factor that undoes the chains' tilts (k_chain):
        //   sigma ~ alpha^_i(m') beta^_{i+1}(m) 2^{(theta'_{i+1} - theta_i)(m' - mean_i)}
        //           2^{(theta'_{i+1} - 1) j} prior R~
        // up to a constant per symbol.  The alpha-side factor is applied in log
        // space and clamped, so a zero alpha never meets an overflowing factor.
        // The per-j factor 2^{phi j}, phi = theta'_{i+1} - 1, splits exactly as
        // 2^{phi (pl + j)} 2^{-phi pl}: folded into the beta window (index pl + j)
        // and the alpha window (index pl).
        for (int idx = threadIdx.x; idx < S * P; idx += blockDim.x) {
            const int il = idx / P, pl = idx - il * P;
            const long long i = ilo + il, p = p0 + pl;
            const long long s = p - (long long)n * i + xmax;
            float v = 0.f;
            if (s >= 0 && s < M && p <= rho) {
                const float a = f.alpha[(size_t)i * f.Mp + s];
                if (a > 0.f) {
                    const double phi = f.thb[i + 1] - 1.0;
                    const float e = (float)((f.thb[i + 1] - f.thf[i]) *
                                                ((double)(s - xmax) - f.mcf[i]) -
                                            phi * (double)pl);
                    v = exp2f(fminf(log2f(a) + e, 126.f));
                }
            }
            Aw[idx] = v;
        }
        for (int idx = threadIdx.x; idx < S * BW; idx += blockDim.x) {
            const int il = idx / BW, k = idx - il * BW;
            const long long i = ilo + il;
            const long long s = p0 - (long long)n * i + xmax - n + k;
            float v = 0.f;
            if (s >= 0 && s < M) {
                const float b = f.beta[(size_t)(i + 1) * f.Mp + s];
                v = b * exp2f((float)(f.thb[i + 1] - 1.0) * (float)k);
            }
            Bw[idx] = v;
        }
        __syncthreads();

        // (C) GEMM over K in chunks.  Micro-tiles 4 rows x 4 columns; when there
        // are fewer micro-tiles than threads the K range is split KS ways.
        const int NRG = S4 / 4, NCG = CW / 4;
        const int NMT = NRG * NCG;
        const int KS = NMT >= (int)blockDim.x ? 1 : (int)blockDim.x / NMT;
        const int slots = NMT * KS;
        const int per_pass = (int)blockDim.x * MT;
        const int npass = (NMT + per_pass - 1) / per_pass;
        for (int pass = 0; pass < npass; ++pass) {
            float acc[MT][4][4];
#pragma unroll
            for (int m = 0; m < MT; ++m)
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[m][r][u] = 0.f;
            for (int kc0 = 0; kc0 < K; kc0 += kKC) {
                const int kn = min(kKC, K - kc0);
                for (int idx = threadIdx.x; idx < kn * S4; idx += blockDim.x) {
                    const int kk = idx / S4, il = idx - kk * S4;
                    const int c = kc0 + kk;
                    const int pl = c / MN, j = c - pl * MN;
                    AB[idx] = (il < S) ? Aw[il * P + pl] * Bw[il * BW + pl + j] : 0.f;
                }
                __syncthreads();
                if (KS > 1) {
                    const int t = threadIdx.x;
                    if (t < slots) {
                        const int mt = t % NMT, ks = t / NMT;
                        const int rg = mt / NCG, cg = mt - rg * NCG;
                        for (int kk = ks; kk < kn; kk += KS) {
                            const float4 a =
                                *reinterpret_cast<const float4 *>(AB + (size_t)kk * S4 + rg * 4);
                            const float4 b = *reinterpret_cast<const float4 *>(
                                Rt + (size_t)(kc0 + kk) * CW + cg * 4);
                            const float av[4] = {a.x, a.y, a.z, a.w};
                            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                            for (int r = 0; r < 4; ++r)
#pragma unroll
                                for (int u = 0; u < 4; ++u)
                                    acc[0][r][u] = fmaf(av[r], bv[u], acc[0][r][u]);
                        }
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < MT; ++m) {
                        const int mt = pass * per_pass + m * (int)blockDim.x + threadIdx.x;
                        if (mt < NMT) {
                            const int rg = mt / NCG, cg = mt - rg * NCG;
                            for (int kk = 0; kk < kn; ++kk) {
                                const float4 a = *reinterpret_cast<const float4 *>(
                                    AB + (size_t)kk * S4 + rg * 4);
                                const float4 b = *reinterpret_cast<const float4 *>(
                                    Rt + (size_t)(kc0 + kk) * CW + cg * 4);
                                const float av[4] = {a.x, a.y, a.z, a.w};
                                const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                                for (int r = 0; r < 4; ++r)
#pragma unroll
                                    for (int u = 0; u < 4; ++u)
                                        acc[m][r][u] = fmaf(av[r], bv[u], acc[m][r][u]);
                            }
                        }
                    }
                }
                __syncthreads();
            }
            if (KS > 1) {
                float *Red = AB;
                if ((int)threadIdx.x < slots) {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            Red[(size_t)threadIdx.x * 16 + r * 4 + u] = acc[0][r][u];
                }
                __syncthreads();
                if ((int)threadIdx.x < NMT) {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            float s = 0.f;
                            for (int ks = 0; ks < KS; ++ks)
                                s += Red[(size_t)(ks * NMT + threadIdx.x) * 16 + r * 4 + u];
                            acc[0][r][u] = s;
                        }
                }
                __syncthreads();
            }
            // (D) owners add into the accumulators / stage tangent sums
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                int mt;
                if (KS > 1) {
                    if (m > 0) break;
                    mt = (int)threadIdx.x;
                } else {
                    mt = pass * per_pass + m * (int)blockDim.x + threadIdx.x;
                }
                if (mt >= NMT) continue;
                const int rg = mt / NCG, cg = mt - rg * NCG;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int il = rg * 4 + r;
                    if (il >= S) break;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int col = cg * 4 + u;
                        const int th = col / DS, D = col - th * DS;
                        if (D >= q) continue;
                        if (th == 0) Lacc[(size_t)(off + il) * q + D] += acc[m][r][u];
                        else Ct[((size_t)(th - 1) * Smax4 + il) * DS + D] = acc[m][r][u];
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
