// Forward producer specialisations for insertion cap I = 1, n = 1..12.
#define MAPDEC_IB 1
#include "producers_inst.cuh"

namespace mdk {

cudaError_t launch_fwd_I1(int n, const FrameDev *frames, const Work *work, int nwork, size_t smem,
                          cudaStream_t st) {
    switch (n) {
        MAPDEC_FOR_N(MAPDEC_CASE_FWD)
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_fwd_tc_I1(int n, const FrameDev *frames, const Work *work, int nwork,
                             size_t smem, cudaStream_t st) {
    switch (n) {
        MAPDEC_FOR_N_TC(MAPDEC_CASE_FWDTC)
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_rmetric_I1(int n, const FrameDev *frame, long long nthreads, cudaStream_t st) {
    switch (n) {
        MAPDEC_FOR_N(MAPDEC_CASE_RM)
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_fwd_ps_I1(int n, const FrameDev *frames, const Work *work, int nwork,
                             cudaStream_t st) {
    switch (n) {
        MAPDEC_FOR_N(MAPDEC_CASE_FWDPS)
        default: return cudaErrorNotSupported;
    }
}

}  // namespace mdk
