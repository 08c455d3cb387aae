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

bool fwd_tc_supported(int q, int n, int I) {
    return specialised(n, I) && n >= 4 && q >= 16 && q <= 64 && q % 16 == 0;
}

size_t fwd_tc_smem_bytes(const FrameDev &f) {
    const size_t MT = ((size_t)f.Pf * f.MN + 127) / 128;
    const size_t NN = ((size_t)f.Sf + 15) & ~(size_t)15;
    const size_t b = (MT * 128 + NN) * (size_t)f.q * 4;  // hi and lo bf16 of both operands
    return b < kTcMinSmem ? kTcMinSmem : b;
}

size_t bwd_tc_smem_bytes(const FrameDev &f) {
    const size_t K = (size_t)f.P * f.MN, Kp = (K + 15) & ~(size_t)15;
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
