#include <algorithm>
// Producers with the run-time (n, I) lattice, plus the (n, I) dispatch.
#include "producers_inst.cuh"

namespace mdk {

cudaError_t launch_fwd_rt(const FrameDev *frames, const Work *work, int nwork, size_t smem,
                          cudaStream_t st) {
    return launch_fwd_t<0, 0>(frames, work, nwork, smem, st);
}
cudaError_t launch_bwd_rt(bool grad, const FrameDev *frames, const Work *work, int nwork,
                          size_t smem, cudaStream_t st) {
    return grad ? launch_bwd_t<0, 0, true>(frames, work, nwork, smem, st)
                : launch_bwd_t<0, 0, false>(frames, work, nwork, smem, st);
}
cudaError_t launch_rmetric_rt(const FrameDev *frame, long long nthreads, cudaStream_t st) {
    return launch_rmetric_t<0, 0>(frame, nthreads, st);
}

// Shared-memory bytes of each producer for frame f.
size_t fwd_smem_bytes(const FrameDev &f) {
    const int S4 = (f.Sf + 3) & ~3;
    const size_t RS = ((size_t)f.Pf * f.MN + 3) & ~(size_t)3;
    return 4 * ((size_t)f.q * RS + (size_t)f.q * S4);
}
size_t bwd_smem_bytes(const FrameDev &f, bool grad) {
    const int NR = grad ? 4 : 1;
    const size_t Smax4 = ((size_t)f.S + 3) & ~(size_t)3;
    const size_t DS = ((size_t)f.q + 3) & ~(size_t)3;
    const size_t K = (size_t)f.P * f.MN;
    const size_t BW = (size_t)f.P + f.MN - 1;
    size_t fl = K * NR * DS + (size_t)f.P * Smax4 + BW * Smax4 + 4 * Smax4 +
                (((size_t)f.S2 * f.q + 3) & ~(size_t)3) +
                (((size_t)f.S2 * 3 + 3) & ~(size_t)3);
    if (grad) fl += 3 * Smax4 * DS;
    return 4 * fl;
}

bool specialised(int n, int I) { return n >= 1 && n <= kMaxSpecN && I >= 1 && I <= 3; }

// ---------------------------------------------------------------------------
// Priors of a frame as the B operand of the W contraction: three bf16 pieces,
// K-major (row = symbol, K = D), the pieces interleaved per 8-row group:
//   byte(i, D, piece) = (i / 8) * 3 kc 128 + piece * kc 128 + (D / 8) * 128
//                       + (i % 8) * 16 + (D % 8) * 2,   kc = q / 8,
// rows up to f.Pgroups * 8 (the rows past N are zero).  A tile's symbols
// [ilo8, ilo8 + NNa) are one contiguous block (a single bulk copy).
// One thread per (8-row group, piece, 8-column chunk, row).
// ---------------------------------------------------------------------------
__global__ void k_prior_split(const FrameDev *__restrict__ frames, int nframes) {
    const int fi = blockIdx.y;
    if (fi >= nframes) return;
    const FrameDev &f = frames[fi];
    if (!f.Pbuf) return;
    const int q = f.q, kc = q >> 3;
    const long long total = (long long)f.Pgroups * kc * 8;  // (group, chunk, row)
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int r8 = (int)(t & 7);
        const long long gc = t >> 3;
        const int c = (int)(gc % kc);
        const long long g = gc / kc;
        const long long i = g * 8 + r8;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = i < f.N ? __ldg(f.priors + i * q + c * 8 + e) : 0.f;
        uint4 p0, p1, p2;
        split3_x8(v, p0, p1, p2);
        unsigned char *base = f.Pbuf + (size_t)g * 3 * kc * 128 + (size_t)c * 128 + r8 * 16;
        *reinterpret_cast<uint4 *>(base) = p0;
        *reinterpret_cast<uint4 *>(base + (size_t)kc * 128) = p1;
        *reinterpret_cast<uint4 *>(base + (size_t)2 * kc * 128) = p2;
    }
}

cudaError_t launch_prior_split(const FrameDev *frames, int nframes, long long max_threads,
                               cudaStream_t st) {
    if (nframes <= 0 || max_threads <= 0) return cudaSuccess;
    int gx = (int)std::min<long long>((max_threads + 255) / 256, 64);
    dim3 grid(std::max(gx, 1), nframes);
    k_prior_split<<<grid, 256, 0, st>>>(frames, nframes);
    return cudaGetLastError();
}

size_t prior_split_bytes(const FrameDev &f) {
    return (size_t)prior_split_groups(f) * 3 * (size_t)(f.q / 8) * 128;
}

int ps_chunk_states(int q, int M) {
    const int c = std::max(1, 2048 / std::max(q, 1));
    return std::min(c, M);
}

size_t bwd_ps_smem_bytes(const FrameDev &f, bool grad) {
    int G = 1;
    while (G * 2 <= f.q && G * 2 <= 32) G *= 2;
    const size_t ngrp = (kThreads / 32) * (32 / G);
    const size_t NR = grad ? 4 : 1;
    const size_t fl = (size_t)f.psC * 4 + ((size_t)f.psC + f.MN - 1) * 4 + 16 +
                      ngrp * (size_t)f.q * NR;
    return 4 * fl;
}

cudaError_t launch_fwd_ps(int n, int I, const FrameDev *frames, const Work *work, int nwork,
                          cudaStream_t st) {
    if (specialised(n, I)) {
        if (I == 1) return launch_fwd_ps_I1(n, frames, work, nwork, st);
        if (I == 2) return launch_fwd_ps_I2(n, frames, work, nwork, st);
        return launch_fwd_ps_I3(n, frames, work, nwork, st);
    }
    return launch_fwd_ps_t<0, 0>(frames, work, nwork, st);
}

cudaError_t launch_bwd_ps(int n, int I, bool grad, const FrameDev *frames, const Work *work,
                          int nwork, size_t smem, cudaStream_t st) {
    if (specialised(n, I)) {
        if (I == 1) return grad ? launch_bwd_ps_I1_grad(n, frames, work, nwork, smem, st)
                                : launch_bwd_ps_I1_plain(n, frames, work, nwork, smem, st);
        if (I == 2) return grad ? launch_bwd_ps_I2_grad(n, frames, work, nwork, smem, st)
                                : launch_bwd_ps_I2_plain(n, frames, work, nwork, smem, st);
        return grad ? launch_bwd_ps_I3_grad(n, frames, work, nwork, smem, st)
                    : launch_bwd_ps_I3_plain(n, frames, work, nwork, smem, st);
    }
    return grad ? launch_bwd_ps_t<0, 0, true>(frames, work, nwork, smem, st)
                : launch_bwd_ps_t<0, 0, false>(frames, work, nwork, smem, st);
}

bool fwd_tc_supported(int q, int n, int I) {
    return specialised(n, I) && n >= 4 && q >= 16 && q <= 64 && q % 16 == 0;
}

size_t fwd_tc_smem_bytes(const FrameDev &f) {
    const size_t MNp = ((size_t)f.MN + 7) & ~(size_t)7;
    const size_t NRa = std::max<size_t>(128, ((size_t)f.Pf * MNp + 7) & ~(size_t)7);
    const size_t NN = ((size_t)f.Sf + 7 + 15) & ~(size_t)15;  // from the 8-aligned first symbol
    const size_t b = (NRa + NN) * (size_t)f.q * 6;           // three bf16 pieces of both operands
    return b < kTcMinSmem ? kTcMinSmem : b;
}

size_t bwd_tc_smem_bytes(const FrameDev &f) {
    const size_t MNp = ((size_t)f.MN + 7) & ~(size_t)7;
    const size_t K = (size_t)f.P * MNp, Kp = (K + 15) & ~(size_t)15;
    const size_t Smax4 = ((size_t)f.S + 3) & ~(size_t)3;
    const size_t BW = (size_t)f.P + f.MN - 1;
    const size_t b = 4 * (size_t)f.q * Kp + 4 * 128 * (size_t)kTcChunkCols +
                     4 * Smax4 * ((size_t)f.P + BW + 4);
    return b < kTcMinSmem ? kTcMinSmem : b;
}

cudaError_t launch_bwd_tc(int n, int I, const FrameDev *frames, const Work *work, int nwork,
                          size_t smem, cudaStream_t st) {
    if (I == 1) return launch_bwd_tc_I1(n, frames, work, nwork, smem, st);
    if (I == 2) return launch_bwd_tc_I2(n, frames, work, nwork, smem, st);
    if (I == 3) return launch_bwd_tc_I3(n, frames, work, nwork, smem, st);
    return cudaErrorNotSupported;
}

cudaError_t launch_fwd_tc(int n, int I, const FrameDev *frames, const Work *work, int nwork,
                          size_t smem, cudaStream_t st) {
    if (I == 1) return launch_fwd_tc_I1(n, frames, work, nwork, smem, st);
    if (I == 2) return launch_fwd_tc_I2(n, frames, work, nwork, smem, st);
    if (I == 3) return launch_fwd_tc_I3(n, frames, work, nwork, smem, st);
    return cudaErrorNotSupported;
}

cudaError_t launch_fwd(int n, int I, const FrameDev *frames, const Work *work, int nwork,
                       size_t smem, cudaStream_t st) {
    if (specialised(n, I)) {
        if (I == 1) return launch_fwd_I1(n, frames, work, nwork, smem, st);
        if (I == 2) return launch_fwd_I2(n, frames, work, nwork, smem, st);
        return launch_fwd_I3(n, frames, work, nwork, smem, st);
    }
    return launch_fwd_rt(frames, work, nwork, smem, st);
}

cudaError_t launch_bwd(int n, int I, bool grad, const FrameDev *frames, const Work *work,
                       int nwork, size_t smem, cudaStream_t st) {
    if (specialised(n, I)) {
        if (I == 1) return launch_bwd_I1(n, grad, frames, work, nwork, smem, st);
        if (I == 2) return launch_bwd_I2(n, grad, frames, work, nwork, smem, st);
        return launch_bwd_I3(n, grad, frames, work, nwork, smem, st);
    }
    return launch_bwd_rt(grad, frames, work, nwork, smem, st);
}

cudaError_t launch_rmetric(int n, int I, const FrameDev *frame, long long nthreads,
                           cudaStream_t st) {
    if (specialised(n, I)) {
        if (I == 1) return launch_rmetric_I1(n, frame, nthreads, st);
        if (I == 2) return launch_rmetric_I2(n, frame, nthreads, st);
        return launch_rmetric_I3(n, frame, nthreads, st);
    }
    return launch_rmetric_rt(frame, nthreads, st);
}

}  // namespace mdk
