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
    const int S4 = (f.S + 3) & ~3;
    const size_t RS = ((size_t)f.P * f.MN + 3) & ~(size_t)3;
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
