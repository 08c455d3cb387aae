// Backward producer specialisations (APP partial sums) for I = 2, n = 1..12.
#define MAPDEC_IB 2
#include "producers_inst.cuh"

namespace mdk {

cudaError_t launch_bwd_I2_plain(int n, const FrameDev *frames, const Work *work, int nwork,
                                  size_t smem, cudaStream_t st) {
    const bool grad = false;
    switch (n) {
        MAPDEC_FOR_N(MAPDEC_CASE_BWDX)
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_bwd_tc_I2(int n, const FrameDev *frames, const Work *work, int nwork,
                             size_t smem, cudaStream_t st) {
    switch (n) {
        MAPDEC_FOR_N_TC(MAPDEC_CASE_BWDTC)
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_bwd_ps_I2_plain(int n, const FrameDev *frames, const Work *work,
                                  int nwork, size_t smem, cudaStream_t st) {
    const bool grad = false;
    switch (n) {
        MAPDEC_FOR_N(MAPDEC_CASE_BWDPS)
        default: return cudaErrorNotSupported;
    }
}

}  // namespace mdk
