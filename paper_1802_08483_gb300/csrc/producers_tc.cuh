// Tensor-core producers (tcgen05).  FP32 accuracy from bf16 operands: an
// operand x is split into bf16 pieces, x = x0 + x1 (+ x2), x_k = bf16 of what
// the earlier pieces left, rounded to nearest, and the product is the sum of
// the piece products of low order, accumulated in FP32 in tensor memory.
//   three pieces, six products (x0 y0, x0 y1, x1 y0, x0 y2, x1 y1, x2 y0): the
//     dropped terms and the representation error are about 2^-24 of each
//     product -- the W contraction, whose errors the recursions carry along
//     the frame;
//   two pieces, three products: about 2^-16 -- the APP contraction, whose
//     error enters each symbol's APP once.
#pragma once

#include "mapdec_kernels.h"
#include "producers.cuh"
#include "tcgen05.cuh"

namespace mdk {

constexpr int kTcCols = 256;  // tensor-memory columns per forward CTA (two CTAs per SM)
constexpr uint32_t kTcWaitLimit = 1u << 26;

__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity) {
    return mbar_wait(bar, parity, kTcWaitLimit);
}

// Two floats rounded to bf16 and packed: a in the low half, b in the high half.
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&t);
}

// 8 consecutive values split into three bf16 pieces, each packed as 8 bf16
// (16 bytes, element e at bits 16 (e % 2) of word e / 2).
__device__ __forceinline__ void split3_x8(const float (&v)[8], uint4 &p0, uint4 &p1, uint4 &p2) {
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float a = v[2 * e], b = v[2 * e + 1];
        uint32_t h = pack_bf16x2(a, b);
        a -= __uint_as_float(h << 16);
        b -= __uint_as_float(h & 0xffff0000u);
        uint32_t m = pack_bf16x2(a, b);
        a -= __uint_as_float(m << 16);
        b -= __uint_as_float(m & 0xffff0000u);
        w0[e] = h;
        w1[e] = m;
        w2[e] = pack_bf16x2(a, b);
    }
    p0 = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    p1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    p2 = make_uint4(w2[0], w2[1], w2[2], w2[3]);
}

// ---------------------------------------------------------------------------
// Tensor-core forward producer: the same work as k_fwd -- the lattices of a
// tile of Pf received positions (eqs. F / F_lastrow) and the prior-weighted
// transition sums W_i(s', j) = sum_D prior_i(D) R[n i + s' - xmax][D][j] (eq.
// gamma summed over D) -- with the contraction over D on the tensor cores:
//     C[m][c] = sum_D R[m][D] prior[ilo8 + c][D],   m = pl * MNp + j,
// MNp = MN rounded up to 8 (rows j >= MN of a position are padding), M = the
// tile's Pf * MNp rows in 128-row tiles, N = NNa symbols starting at the
// 8-aligned ilo8 <= ilo (a multiple of 16, at most 256), K = q.  Three
// pieces, six products.
// Shared memory: R, 3 pieces, MN-major (M contiguous in the 16-byte rows of a
// core matrix: byte(m, D) = (D / 8) (MT 128 / 8) 128 + (m / 8) 128 + (D % 8) 16
// + (m % 8) 2), so a lattice thread stores 8 consecutive lengths j as one
// 16-byte vector per piece; then the priors block, bulk-copied from f.Pbuf
// during the lattices.  Rows that hold no data only feed outputs that are not
// stored.  Tensor memory: 256 columns, two accumulators of 128 when NNa <= 128
// (the next M-tile's MMAs overlap this one's epilogue), else one.  Every CTA
// that allocates tensor memory frees it before it exits; every wait is
// bounded (ST_TIMEOUT).
// ---------------------------------------------------------------------------
template <int NB, int IB>
__global__ void __launch_bounds__(kThreads, 2) k_fwd_tc(const FrameDev *__restrict__ frames,
                                                        const Work *__restrict__ work) {
    static_assert(NB > 0, "compile-time lattice only");
    constexpr int n = NB;
    constexpr int MN = NB * (IB + 1) + 1;
    constexpr int MNp = (MN + 7) & ~7;
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    const int q = f.q, P = f.Pf, M = f.M, xmax = f.xmax;
    const long long rho = f.rho;
    const long long p0 = (long long)wk.tile * P;
    int ilo, ihi;
    tile_symbols(f, wk.tile, ilo, ihi);
    if (ihi < ilo) return;  // uniform over the CTA, before any tensor memory is held
    const int ilo8 = ilo & ~7;
    const int NNa = (ihi - ilo8 + 1 + 15) & ~15;
    const int NR = P * MNp;
    const int MT = (NR + 127) >> 7;
    // rows held in shared memory: NR rounded up to 8, at least one M-tile.  The
    // last M-tile starts at NRa - 128 (overlapping the one before when NR is
    // not a multiple of 128) and stores only the rows past the earlier tiles.
    const int NRa = max(128, (NR + 7) & ~7);
    const int mg = NRa >> 3;  // 8-row groups of the R operand
    auto mt0 = [&](int t) { return min(t * 128, NRa - 128); };
    const int kc = q >> 3;
    const int nbuf = NNa <= 128 ? 2 : 1;
    const uint32_t pbytes = (uint32_t)(NNa >> 3) * 3u * (uint32_t)kc * 128u;

    extern __shared__ __align__(128) unsigned char tsm[];
    unsigned char *R0 = tsm;  // piece k at R0 + k * NRa q 2
    const size_t rpiece = (size_t)NRa * q * 2;
    unsigned char *Pb = R0 + 3 * rpiece;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[3];  // [0], [1]: MMA accumulators; [2]: priors copy
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(&s_tmem, kTcCols);
    if (tid == 0) {
        s_fail = 0;
        for (int b = 0; b < 3; ++b) mbar_init(&s_bar[b], 1);
        fence_mbar_init();
        // the tile's priors block: groups ilo8/8 .. ilo8/8 + NNa/8 - 1 of f.Pbuf
        mbar_expect_tx(&s_bar[2], pbytes);
        bulk_g2s(Pb, f.Pbuf + (size_t)(ilo8 >> 3) * 3 * kc * 128, pbytes, &s_bar[2]);
    }

    // (A) lattices: a warp covers 4 positions x 8 codewords; a quarter warp
    // (one position, 8 codewords) stores 128 contiguous bytes per chunk
    const int nblk = ((P + 3) >> 2) * (q >> 3);
    for (int b = warp; b < nblk; b += kThreads / 32) {
        const int pb = b / (q >> 3), db = b - pb * (q >> 3);
        const int pl = pb * 4 + (lane >> 3), D = db * 8 + (lane & 7);
        if (pl >= P) continue;
        const long long p = p0 + pl;
        float v[MNp];
        if (p <= rho) {
            eval_metric<NB, IB, 0>(f, p, D, v);
        } else {
#pragma unroll
            for (int j = 0; j < MN; ++j) v[j] = 0.f;
        }
#pragma unroll
        for (int j = MN; j < MNp; ++j) v[j] = 0.f;
        const uint32_t dbase = (uint32_t)(D >> 3) * (uint32_t)mg * 128u + (uint32_t)(D & 7) * 16u;
#pragma unroll
        for (int c = 0; c < MNp / 8; ++c) {
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = v[c * 8 + e];
            uint4 a0, a1, a2;
            split3_x8(x, a0, a1, a2);
            const uint32_t o = dbase + (uint32_t)((pl * MNp + c * 8) >> 3) * 128u;
            *reinterpret_cast<uint4 *>(R0 + o) = a0;
            *reinterpret_cast<uint4 *>(R0 + rpiece + o) = a1;
            *reinterpret_cast<uint4 *>(R0 + 2 * rpiece + o) = a2;
        }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = tc::idesc_bf16(128, NNa) | (1u << 15);  // A MN-major

    // MMAs of M-tile t into accumulator t % nbuf (one thread).  The operands of
    // one MMA differ from the first one's only in their start addresses, which
    // sit in the descriptors' low field (address / 16, below 2^14: no carry), so
    // the descriptors are formed once and offset per MMA.
    const uint64_t da0 = tc::smem_desc_mn(smem_u32(R0), (uint32_t)mg);
    const uint64_t db0 = tc::smem_desc_kmajor(smem_u32(Pb), 3u * (uint32_t)kc);
    const uint32_t a_piece = (uint32_t)(rpiece >> 4), a_kstep = (uint32_t)mg * 16u;  // 16-byte units
    const uint32_t b_piece = (uint32_t)kc * 8u;
    auto issue = [&](int t) {
        if constexpr (IB <= 2) {
            const uint32_t d = tmem + (uint32_t)((t % nbuf) * 128);
            const uint64_t da_t = da0 + (uint64_t)(mt0(t) >> 3) * 8u;  // 128 bytes per 8-row group
            uint32_t ak = 0, bk = 0;
            for (int k0 = 0; k0 < q; k0 += 16, ak += a_kstep, bk += 16u) {
                const uint64_t da = da_t + ak, db = db0 + bk;
                // pieces (A, B): (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
                tc::mma_bf16(d, da, db, idesc, k0 > 0 ? 1u : 0u);
                tc::mma_bf16(d, da, db + b_piece, idesc, 1u);
                tc::mma_bf16(d, da + a_piece, db, idesc, 1u);
                tc::mma_bf16(d, da, db + 2u * b_piece, idesc, 1u);
                tc::mma_bf16(d, da + a_piece, db + b_piece, idesc, 1u);
                tc::mma_bf16(d, da + 2u * a_piece, db, idesc, 1u);
            }
            tc::commit(&s_bar[t % nbuf]);
        } else {
            // longer lattices (I = 3): descriptors formed per MMA (the kernel
            // spills less this way; measured on the N = 8000 workload)
            const uint32_t d = tmem + (uint32_t)((t % nbuf) * 128);
            const uint32_t rb = smem_u32(R0) + (uint32_t)(mt0(t) >> 3) * 128u;
            const uint32_t pbs = smem_u32(Pb);
            const int pa[6] = {0, 0, 1, 0, 1, 2}, pp[6] = {0, 1, 0, 2, 1, 0};
            for (int k0 = 0; k0 < q; k0 += 16) {
#pragma unroll
                for (int pr = 0; pr < 6; ++pr) {
                    const uint32_t a = rb + (uint32_t)pa[pr] * (uint32_t)rpiece +
                                       (uint32_t)(k0 >> 3) * (uint32_t)mg * 128u;
                    const uint32_t bsm = pbs + (uint32_t)pp[pr] * (uint32_t)kc * 128u +
                                         (uint32_t)(k0 >> 3) * 128u;
                    tc::mma_bf16(d, tc::smem_desc_mn(a, (uint32_t)mg),
                                 tc::smem_desc_kmajor(bsm, 3u * (uint32_t)kc), idesc,
                                 (k0 > 0 || pr > 0) ? 1u : 0u);
                }
            }
            tc::commit(&s_bar[t % nbuf]);
        }
    };
    if (tid == 0) {
        if (!tc_wait(&s_bar[2], 0)) s_fail = ST_TIMEOUT;  // the priors block has landed
        tc::fence_after_sync();
        if (!s_fail)
            for (int t = 0; t < nbuf && t < MT; ++t) issue(t);
    }
    __syncthreads();
    const bool issued = !s_fail;

    // (C) epilogue per M-tile: TMEM lane = row m of the tile, 16 columns per
    // load; the two warpgroups take alternate 16-column chunks.  For one symbol
    // the valid rows of a warp are runs of consecutive floats of W (MNS == MN).
    const int lg = warp & 3, half = warp >> 2;
    for (int t = 0; t < MT && issued; ++t) {
        const int buf = t % nbuf;
        // one thread waits for the MMAs (bounded); the others wait at the CTA
        // barrier, which takes no issue slots from the co-resident CTA
        if (tid == 0 && !tc_wait(&s_bar[buf], (uint32_t)((t / nbuf) & 1))) s_fail = ST_TIMEOUT;
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        const int m = mt0(t) + lg * 32 + lane;
        const int pl = m / MNp, j = m - pl * MNp;
        const long long p = p0 + pl;
        // this row's symbols: drift state s = p + xmax - n i inside [0, M), so
        // i in [ceil((p + xmax - M + 1) / n), floor((p + xmax) / n)], within the tile's
        const long long pw = p + xmax;
        int clo = (int)max((long long)ilo, ceildiv(pw - M + 1, n)) - ilo8;
        int chi = (int)min((long long)ihi, floordiv(pw, n)) - ilo8;
        // nothing to store (or stored by the M-tile before, which this one overlaps)
        if (!(pl < P && j < MN && p <= rho) || m < t * 128 || s_fail) chi = -1;
        // W[i][s][j] = W + pw MNS + j + i (wblk - n MNS)
        float *wrow = f.W + (size_t)pw * f.MNS + j + (size_t)ilo8 * (f.wblk - (long long)n * f.MNS);
        const long long wstep = f.wblk - (long long)n * f.MNS;
        const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(buf * 128);
        for (int c0 = half * 16; c0 < NNa; c0 += 32) {
            float v[16];
            tc::ld16(ta + (uint32_t)c0, v);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int c = c0 + e;
                if (c >= clo && c <= chi) wrow[(long long)c * wstep] = v[e];
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0 && t + nbuf < MT) {
            tc::fence_after_sync();
            issue(t + nbuf);
        }
    }
    if (tid == 0 && s_fail) atomicMax(f.status, s_fail);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTcCols);
}

}  // namespace mdk

namespace mdk {

// ---------------------------------------------------------------------------
// Tensor-core APP producer (decode mode).  Same work item and output as k_bwd
// (a super-tile of nsub sub-tiles of P positions; Lp rows of the super-tile's
// symbols), with the contraction of eqs. (L), (sigma) on the tensor cores:
//     C[il2][D] += sum_k A[il2][k] R[D][k],   k = pl * MNp + j,
//     A[il2][k] = Aw[pl][il] Bw[pl + j][il]   (il = il2 - off: the sub-tile's
//                                              symbols; other rows zero)
// with MNp = MN rounded up to 8 (lengths j >= MN are zero columns of both
// operands), accumulated over every sub-tile in one TMEM accumulator of 128
// lanes (il2 < S2 <= 128) and q columns.  Two bf16 pieces, three products.
// Shared memory: R, 2 pieces, K-major [q rows][Kp] (Kp = P MNp rounded up to
// 16, the pad columns zero): a lattice thread stores 8 consecutive lengths as
// one 16-byte row of a core matrix per piece; A, 2 pieces, [128 rows][kTcChunk],
// built chunk by chunk, 8 columns (one position) per thread and row, and read
// by the MMAs before the next chunk is built; the windows Aw, Bw (FP32) and the
// per-symbol tilt constants.
// ---------------------------------------------------------------------------
constexpr int kTcChunk = kTcChunkCols;  // A-operand columns per chunk (a multiple of 16)

// 8 values split into two bf16 pieces, each packed as 8 bf16 (16 bytes).
__device__ __forceinline__ void split2_x8(const float (&v)[8], uint4 &p0, uint4 &p1) {
    uint32_t w0[4], w1[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float a = v[2 * e], b = v[2 * e + 1];
        const uint32_t h = pack_bf16x2(a, b);
        a -= __uint_as_float(h << 16);
        b -= __uint_as_float(h & 0xffff0000u);
        w0[e] = h;
        w1[e] = pack_bf16x2(a, b);
    }
    p0 = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    p1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
}

template <int NB, int IB>
__global__ void __launch_bounds__(kThreads, 2) k_bwd_tc(const FrameDev *__restrict__ frames,
                                                        const Work *__restrict__ work) {
    static_assert(NB > 0, "compile-time lattice only");
    constexpr int n = NB;
    constexpr int MN = NB * (IB + 1) + 1;
    constexpr int MNp = (MN + 7) & ~7;
    const Work wk = work[blockIdx.x];
    const FrameDev &f = frames[wk.frame];
    const int q = f.q, P = f.P;
    const long long rho = f.rho;
    int ilo2, ihi2;
    super_symbols(f, wk.tile, ilo2, ihi2);
    const int S2 = ihi2 - ilo2 + 1;
    if (S2 <= 0) return;  // uniform over the CTA, before any tensor memory is held
    const int Kp = (P * MNp + 15) & ~15;
    const int kcR = Kp >> 3;
    constexpr int kcA = kTcChunk >> 3;
    const int BW = P + MN - 1;
    const int Smax4 = (f.S + 3) & ~3;
    const uint32_t ncols = q <= 32 ? 32u : 64u;
    const size_t rpiece = (size_t)q * Kp * 2, apiece = (size_t)128 * kTcChunk * 2;

    extern __shared__ __align__(128) unsigned char tsm[];
    unsigned char *R0 = tsm;  // pieces at R0, R0 + rpiece
    unsigned char *A0 = R0 + 2 * rpiece;  // pieces at A0, A0 + apiece
    float *Aw = reinterpret_cast<float *>(A0 + 2 * apiece);
    float *Bw = Aw + (size_t)P * Smax4;
    int *symE = reinterpret_cast<int *>(Bw + (size_t)BW * Smax4);
    float *symF = reinterpret_cast<float *>(symE + Smax4);
    float *symG = symF + Smax4;
    float *symPhi = symG + Smax4;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(&s_tmem, ncols);
    if (tid == 0) {
        s_fail = 0;
        mbar_init(&s_bar, 1);
        fence_mbar_init();
    }
    // the pad columns P MNp .. Kp-1 of R stay zero (the lattices write below them)
    for (int e = tid; e < q * ((Kp - P * MNp) >> 3); e += kThreads) {
        const int per = (Kp - P * MNp) >> 3;
        const int D = e / per, g = P * MNp / 8 + e % per;
        const uint32_t o = tc::op_offset(D, g * 8, kcR);
        *reinterpret_cast<uint4 *>(R0 + o) = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(R0 + rpiece + o) = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = tc::idesc_bf16(128, q);

    uint32_t phase = 0;
    bool pending = false;  // MMAs committed and not yet waited for
    bool issued = false;   // the accumulator holds data
    auto drain = [&]() {
        if (pending) {
            // one thread waits (bounded); the others at the CTA barrier
            if (tid == 0 && !tc_wait(&s_bar, phase)) s_fail = ST_TIMEOUT;
            tc::fence_before_sync();
            __syncthreads();
            phase ^= 1u;
            pending = false;
            tc::fence_after_sync();
        }
    };

    for (int sub = 0; sub < f.nsub; ++sub) {
        const long long p0 = ((long long)wk.tile * f.nsub + sub) * P;
        if (p0 > rho) break;
        int ilo, ihi;
        range_symbols(f, p0, p0 + P - 1, ilo, ihi);
        const int S = ihi - ilo + 1;
        if (S <= 0) continue;
        const int S4 = (S + 3) & ~3;
        const int off = ilo - ilo2;

        window_constants(f, p0, n, ilo, S, S4, symE, symF, symG, symPhi);
        window_fetch(f, p0, n, ilo, S, S4, P, BW, Aw, Bw);
        drain();  // the previous sub-tile's MMAs have read R and A

        // (A) lattices into R: a warp covers 4 positions x 8 codewords; a quarter
        // warp (one position) stores 8 consecutive 16-byte rows of a core matrix
        const int nblk = ((P + 3) >> 2) * (q >> 3);
        for (int b = warp; b < nblk; b += kThreads / 32) {
            const int pb = b / (q >> 3), db = b - pb * (q >> 3);
            const int pl = pb * 4 + (lane >> 3), D = db * 8 + (lane & 7);
            if (pl >= P) continue;
            const long long p = p0 + pl;
            float v[MNp];
            if (p <= rho) {
                eval_metric<NB, IB, 0>(f, p, D, v);
            } else {
#pragma unroll
                for (int j = 0; j < MN; ++j) v[j] = 0.f;
            }
#pragma unroll
            for (int j = MN; j < MNp; ++j) v[j] = 0.f;
#pragma unroll
            for (int c = 0; c < MNp / 8; ++c) {
                float x[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] = v[c * 8 + e];
                uint4 a0, a1;
                split2_x8(x, a0, a1);
                const uint32_t o = tc::op_offset(D, pl * MNp + c * 8, kcR);
                *reinterpret_cast<uint4 *>(R0 + o) = a0;
                *reinterpret_cast<uint4 *>(R0 + rpiece + o) = a1;
            }
        }
        cp_async_wait_all();
        __syncthreads();
        window_tilt(S, S4, P, BW, Aw, Bw, symE, symF, symG, symPhi);
        __syncthreads();

        // (C) A chunk by chunk: a thread builds the 8 columns of one position
        // (one 16-byte store per piece); a warp covers 32 consecutive rows
        const int kdata = P * MNp;  // columns holding positions; the rest stay zero
        for (int c0 = 0; c0 < Kp; c0 += kTcChunk) {
            const int w = min(kTcChunk, Kp - c0);
            drain();  // the previous chunk's MMAs have read A
            for (int u = tid; u < 128 * (w >> 3); u += kThreads) {
                const int il2 = u & 127, g = u >> 7;
                const int il = il2 - off;
                const int k0 = c0 + g * 8;
                uint4 a0 = make_uint4(0u, 0u, 0u, 0u), a1 = a0;
                if (il >= 0 && il < S && k0 < kdata) {
                    const int pl = k0 / MNp, j0 = k0 - pl * MNp;
                    const float aw = Aw[pl * S4 + il];
                    if (aw != 0.f) {
                        float x[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int j = j0 + e;
                            x[e] = j < MN ? aw * Bw[(pl + j) * S4 + il] : 0.f;
                        }
                        split2_x8(x, a0, a1);
                    }
                }
                const uint32_t o = tc::op_offset(il2, g * 8, kcA);
                *reinterpret_cast<uint4 *>(A0 + o) = a0;
                *reinterpret_cast<uint4 *>(A0 + apiece + o) = a1;
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                // descriptors formed once, offset per K step (start address / 16 in
                // their low field, below 2^14)
                const uint64_t dah = tc::smem_desc(smem_u32(A0), kcA);
                const uint64_t dal = dah + (uint64_t)(apiece >> 4);
                const uint64_t drh = tc::smem_desc(smem_u32(R0), kcR) + (uint64_t)((c0 >> 3) * 8);
                const uint64_t drl = drh + (uint64_t)(rpiece >> 4);
                for (int k0 = 0; k0 < w; k0 += 16) {
                    const uint64_t o = (uint64_t)((k0 >> 3) * 8);  // 128 bytes per 8-column chunk
                    tc::mma_bf16(tmem, dah + o, drh + o, idesc, issued ? 1u : 0u);
                    issued = true;
                    tc::mma_bf16(tmem, dah + o, drl + o, idesc, 1u);
                    tc::mma_bf16(tmem, dal + o, drh + o, idesc, 1u);
                }
                tc::commit(&s_bar);
            }
            issued = true;  // every thread tracks it (uniform)
            pending = true;
        }
    }
    drain();

    // (D) the super-tile's sums: TMEM lane il2, columns D, 16 per load; the two
    // warpgroups take alternate 16-column chunks.  No MMA ran: zeros.
    const size_t row0 = (size_t)wk.tile * f.S2;
    const int lg = warp & 3, half = warp >> 2;
    const int il2 = lg * 32 + lane;
    const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16);
    for (int c0 = half * 16; c0 < q; c0 += 32) {
        float v[16];
        if (issued) {
            tc::ld16(ta + (uint32_t)c0, v);
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = 0.f;
        }
        if (il2 < S2 && !s_fail) {
            float *dst = f.Lp + (row0 + il2) * q + c0;
#pragma unroll
            for (int e = 0; e < 16; ++e) dst[e] = v[e];
        }
    }
    if (tid == 0 && s_fail) atomicMax(f.status, s_fail);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

}  // namespace mdk
