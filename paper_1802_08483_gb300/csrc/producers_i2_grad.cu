// Backward producer specialisations with tangents (gradient mode) for I = 2, n = 1..12.
#define MAPDEC_IB 2
#include "producers_inst.cuh"

namespace mdk {

cudaError_t launch_bwd_I2_grad(int n, const FrameDev *frames, const Work *work, int nwork,
                                 size_t smem, cudaStream_t st) {
    const bool grad = true;
    switch (n) {
        MAPDEC_FOR_N(MAPDEC_CASE_BWDX)
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_bwd_I2(int n, bool g, const FrameDev *frames, const Work *work, int nwork,
                          size_t smem, cudaStream_t st) {
    return g ? launch_bwd_I2_grad(n, frames, work, nwork, smem, st)
             : launch_bwd_I2_plain(n, frames, work, nwork, smem, st);
}

cudaError_t launch_bwd_ps_I2_grad(int n, const FrameDev *frames, const Work *work,
                                  int nwork, size_t smem, cudaStream_t st) {
    const bool grad = true;
    switch (n) {
        MAPDEC_FOR_N(MAPDEC_CASE_BWDPS)
        default: return cudaErrorNotSupported;
    }
}

}  // namespace mdk
