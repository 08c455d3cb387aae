// Producers for frames with one codebook per symbol (the constituent
// encodings C_i of Sec. II-A; eq. (gamma) takes C_i(D)).  The receiver metric
// of symbol i then depends on (i, m', D), not only on the received position
// p = n i + m', so the lattices run on the paper's (i, m', D) grid (no
// position dedupe).  One CTA per (frame, symbol i, chunk of psC start states
// s' = m' + xmax); work item tile = i * psT + chunk.
//
//   k_fwd_ps : W_i(s', j) = sum_D prior_i(D) R(Y[p .. p+j) | C_i(D))
//   k_bwd_ps : the APP numerator of eq. (L) without the prior,
//              sum_{s', j} alpha_i(s') R(.. | C_i(D)) beta_{i+1}(s' + j - n)
//              (with the chains' tilt factors), one partial row per work item
//              (Lp row = tile); in gradient mode also the tangent sums
//              sum_D prior_i(D) (the same with dR/dtheta), Gp row = tile.
//
// Lanes: groups of G lanes (G = the largest power of two <= min(q, 32)) take
// the codewords D = lane, lane + G, ... of one start state; the groups of a
// warp take consecutive states.  Sums over D combine by shuffles inside a
// group (fwd) or through shared memory across groups (bwd), in a fixed order.
#pragma once

#include "producers.cuh"

namespace mdk {

__device__ __forceinline__ int ps_group_lanes(int q) {
    int g = 1;
    while (g * 2 <= q && g * 2 <= 32) g *= 2;
    return g;
}

// Lattice (p, x) with an explicit codeword; out[j] for j < MN, zero past rho.
template <int NB, int IB, int MODE>
__device__ __forceinline__ void eval_metric_x(const FrameDev &f, long long p, uint32_t x,
                                              float *out) {
    const int MN = (NB == 0) ? f.MN : NB * (IB + 1) + 1;
    float F[kMaxMN], T[kMaxMN];
    const uint64_t y = rx_window(f.rxbits, p);
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

template <int NB, int IB>
__global__ void __launch_bounds__(kThreads) k_fwd_ps(const FrameDev *__restrict__ frames,
                                                     const Work *__restrict__ work) {
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    const int n = (NB == 0) ? f.n : NB;
    constexpr int MNC = (NB == 0) ? kMaxMN : NB * (IB + 1) + 1;
    const int MN = (NB == 0) ? f.MN : MNC;
    const int q = f.q, M = f.M, xmax = f.xmax;
    const int i = wk.tile / f.psT, c = wk.tile - i * f.psT;
    const int s0 = c * f.psC, s1 = min(M, s0 + f.psC);
    const uint32_t *cwi = f.cw + (size_t)i * q;
    const float *pri = f.priors + (size_t)i * q;
    float *Wi = f.W + (size_t)i * f.wblk;
    const int G = ps_group_lanes(q);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gpw = 32 / G, ngrp = (kThreads / 32) * gpw;
    const int grp = warp * gpw + lane / G, gl = lane & (G - 1);
    for (int sb = s0; sb < s1; sb += ngrp) {  // uniform trip count over the CTA
        const int s = sb + grp;
        const long long p = (long long)n * i + s - xmax;
        const bool valid = s < s1 && p >= 0 && p <= f.rho;
        float acc[MNC];
#pragma unroll
        for (int j = 0; j < MNC; ++j) acc[j] = 0.f;
        if (valid) {
            for (int D = gl; D < q; D += G) {
                float v[kMaxMN];
                eval_metric_x<NB, IB, 0>(f, p, __ldg(cwi + D), v);
                const float w = __ldg(pri + D);
#pragma unroll
                for (int j = 0; j < MNC; ++j)
                    if (j < MN) acc[j] = fmaf(w, v[j], acc[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < MNC; ++j) {
            if (j < MN) {
                for (int o = G >> 1; o > 0; o >>= 1)
                    acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
            }
        }
        if (valid && gl == 0) {
#pragma unroll
            for (int j = 0; j < MNC; ++j)
                if (j < MN) Wi[(size_t)s * f.MNS + j] = acc[j];
        }
    }
}

// smem: Aw[psC][4], Bw[psC + MN - 1][4] (the windows of one symbol, row
// stride 4), 4 x 4 tilt constants, red[ngrp][q][NR] (per-group sums).
template <int NB, int IB, bool GRAD>
__global__ void __launch_bounds__(kThreads) k_bwd_ps(const FrameDev *__restrict__ frames,
                                                     const Work *__restrict__ work) {
    constexpr int NR = GRAD ? 4 : 1;
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    const int n = (NB == 0) ? f.n : NB;
    constexpr int MNC = (NB == 0) ? kMaxMN : NB * (IB + 1) + 1;
    const int MN = (NB == 0) ? f.MN : MNC;
    const int q = f.q, M = f.M, xmax = f.xmax;
    const int i = wk.tile / f.psT, c = wk.tile - i * f.psT;
    const int s0 = c * f.psC, s1 = min(M, s0 + f.psC);
    const int P = s1 - s0, BW = P + MN - 1;
    const long long p0 = (long long)n * i + s0 - xmax;  // position of state s0
    const uint32_t *cwi = f.cw + (size_t)i * q;
    const int G = ps_group_lanes(q);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gpw = 32 / G, ngrp = (kThreads / 32) * gpw;
    const int grp = warp * gpw + lane / G, gl = lane & (G - 1);

    extern __shared__ float4 psm4[];
    float *Aw = reinterpret_cast<float *>(psm4);
    float *Bw = Aw + (size_t)f.psC * 4;
    int *symE = reinterpret_cast<int *>(Bw + (size_t)(f.psC + MN - 1) * 4);
    float *symF = reinterpret_cast<float *>(symE + 4);
    float *symG = symF + 4;
    float *symPhi = symG + 4;
    float *red = symPhi + 4;  // [ngrp][q][NR]

    window_constants(f, p0, n, i, 1, 4, symE, symF, symG, symPhi);
    window_fetch(f, p0, n, i, 1, 4, P, BW, Aw, Bw);
    cp_async_wait_all();
    __syncthreads();
    window_tilt(1, 4, P, BW, Aw, Bw, symE, symF, symG, symPhi);
    __syncthreads();

    // per thread: its codewords D = gl + G r, summed over its states
    const int nr = (q - gl + G - 1) / G;  // codewords of this lane
    for (int r = 0; r < nr; ++r) {
        const int D = gl + G * r;
        float cs[NR];
#pragma unroll
        for (int t = 0; t < NR; ++t) cs[t] = 0.f;
        for (int sb = s0; sb < s1; sb += ngrp) {
            const int s = sb + grp;
            const int sl = s - s0;
            const long long p = p0 + sl;
            if (s >= s1 || p < 0 || p > f.rho) continue;
            const float a = Aw[sl * 4];
            if (a == 0.f) continue;
            const uint32_t x = __ldg(cwi + D);
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                float v[kMaxMN];
                if (t == 0) eval_metric_x<NB, IB, 0>(f, p, x, v);
                if (GRAD && t == 1) eval_metric_x<NB, IB, 1>(f, p, x, v);
                if (GRAD && t == 2) eval_metric_x<NB, IB, 2>(f, p, x, v);
                if (GRAD && t == 3) eval_metric_x<NB, IB, 3>(f, p, x, v);
                float dot = 0.f;
#pragma unroll
                for (int j = 0; j < MNC; ++j)
                    if (j < MN) dot = fmaf(Bw[(sl + j) * 4], v[j], dot);
                cs[t] = fmaf(a, dot, cs[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < NR; ++t) red[((size_t)grp * q + D) * NR + t] = cs[t];
    }
    __syncthreads();
    // sums over the groups in group order, then (gradient mode) prior-weighted
    // sums over D of the tangent rows
    for (int e = threadIdx.x; e < q * NR; e += kThreads) {
        const int D = e / NR, t = e - D * NR;
        float s = 0.f;
        for (int g = 0; g < ngrp; ++g) s += red[((size_t)g * q + D) * NR + t];
        red[e] = s;  // row 0 of red now holds the CTA's sums (group 0's entries were read first)
    }
    __syncthreads();
    for (int D = threadIdx.x; D < q; D += kThreads) f.Lp[(size_t)wk.tile * q + D] = red[D * NR];
    if (GRAD && warp == 0) {
        const float *pri = f.priors + (size_t)i * q;
        for (int t = 1; t < NR; ++t) {
            float s = 0.f;
            for (int D = lane; D < q; D += 32) s = fmaf(__ldg(pri + D), red[D * NR + t], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) f.Gp[(size_t)wk.tile * 3 + (t - 1)] = s;
        }
    }
}

}  // namespace mdk
