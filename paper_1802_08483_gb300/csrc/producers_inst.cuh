// Launch templates for one (n, I) specialisation of the producers.
#pragma once

#include "mapdec_kernels.h"
#include "producers.cuh"
#include "producers_ps.cuh"
#include "producers_tc.cuh"

namespace mdk {

template <int NB, int IB>
cudaError_t launch_fwd_t(const FrameDev *fr, const Work *w, int nw, size_t smem, cudaStream_t st) {
    // I >= 3: the 128-register build (two CTAs per SM)
    auto kern = [] {
        if constexpr (IB >= 3) return k_fwd_occ2<NB, IB>;
        else return k_fwd<NB, IB>;
    }();
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = smem_optin_once(kern, attr);
    if (e != cudaSuccess) return e;
    if (nw <= 0) return cudaSuccess;
    kern<<<nw, kThreads, smem, st>>>(fr, w);
    return cudaGetLastError();
}

template <int NB, int IB, bool GRAD>
cudaError_t launch_bwd_t(const FrameDev *fr, const Work *w, int nw, size_t smem, cudaStream_t st) {
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = smem_optin_once(k_bwd<NB, IB, GRAD>, attr);
    if (e != cudaSuccess) return e;
    if (nw <= 0) return cudaSuccess;
    k_bwd<NB, IB, GRAD><<<nw, kThreads, smem, st>>>(fr, w);
    return cudaGetLastError();
}

// Tensor-core forward producer (q a multiple of 16, n >= 4: see producers_tc.cuh).
template <int NB, int IB>
cudaError_t launch_fwd_tc_t(const FrameDev *fr, const Work *w, int nw, size_t smem,
                            cudaStream_t st) {
    if constexpr (NB >= 4) {
        static std::atomic<uint64_t> attr{0};
        cudaError_t e = smem_optin_once(k_fwd_tc<NB, IB>, attr);
        if (e != cudaSuccess) return e;
        if (nw <= 0) return cudaSuccess;
        k_fwd_tc<NB, IB><<<nw, kThreads, smem, st>>>(fr, w);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

// Tensor-core APP producer, decode mode (producers_tc.cuh).
template <int NB, int IB>
cudaError_t launch_bwd_tc_t(const FrameDev *fr, const Work *w, int nw, size_t smem,
                            cudaStream_t st) {
    if constexpr (NB >= 4) {
        static std::atomic<uint64_t> attr{0};
        cudaError_t e = smem_optin_once(k_bwd_tc<NB, IB>, attr);
        if (e != cudaSuccess) return e;
        if (nw <= 0) return cudaSuccess;
        k_bwd_tc<NB, IB><<<nw, kThreads, smem, st>>>(fr, w);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

// Per-symbol-codebook producers (producers_ps.cuh).
template <int NB, int IB>
cudaError_t launch_fwd_ps_t(const FrameDev *fr, const Work *w, int nw, cudaStream_t st) {
    if (nw <= 0) return cudaSuccess;
    k_fwd_ps<NB, IB><<<nw, kThreads, 0, st>>>(fr, w);
    return cudaGetLastError();
}
template <int NB, int IB, bool GRAD>
cudaError_t launch_bwd_ps_t(const FrameDev *fr, const Work *w, int nw, size_t smem,
                            cudaStream_t st) {
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = smem_optin_once(k_bwd_ps<NB, IB, GRAD>, attr);
    if (e != cudaSuccess) return e;
    if (nw <= 0) return cudaSuccess;
    k_bwd_ps<NB, IB, GRAD><<<nw, kThreads, smem, st>>>(fr, w);
    return cudaGetLastError();
}

template <int NB, int IB>
cudaError_t launch_rmetric_t(const FrameDev *fr, long long nthreads, cudaStream_t st) {
    if (nthreads <= 0) return cudaSuccess;
    const long long blocks = (nthreads + kThreads - 1) / kThreads;
    k_rmetric<NB, IB><<<(unsigned)blocks, kThreads, 0, st>>>(fr);
    return cudaGetLastError();
}

}  // namespace mdk

// Per-I dispatch over n = 1..12.
#define MAPDEC_CASE_FWD(NV) case NV: return launch_fwd_t<NV, MAPDEC_IB>(frames, work, nwork, smem, st);
#define MAPDEC_CASE_BWD(NV)                                                            \
    case NV:                                                                           \
        return grad ? launch_bwd_t<NV, MAPDEC_IB, true>(frames, work, nwork, smem, st) \
                    : launch_bwd_t<NV, MAPDEC_IB, false>(frames, work, nwork, smem, st);
// grad is a compile-time constant in each unit, so only one variant is instantiated
#define MAPDEC_CASE_BWDX(NV) \
    case NV: return launch_bwd_t<NV, MAPDEC_IB, grad>(frames, work, nwork, smem, st);
#define MAPDEC_CASE_RM(NV) case NV: return launch_rmetric_t<NV, MAPDEC_IB>(frame, nthreads, st);
#define MAPDEC_CASE_FWDTC(NV) case NV: return launch_fwd_tc_t<NV, MAPDEC_IB>(frames, work, nwork, smem, st);
#define MAPDEC_CASE_BWDTC(NV) case NV: return launch_bwd_tc_t<NV, MAPDEC_IB>(frames, work, nwork, smem, st);
#define MAPDEC_CASE_FWDPS(NV) case NV: return launch_fwd_ps_t<NV, MAPDEC_IB>(frames, work, nwork, st);
#define MAPDEC_CASE_BWDPS(NV) case NV: return launch_bwd_ps_t<NV, MAPDEC_IB, grad>(frames, work, nwork, smem, st);
#define MAPDEC_FOR_N_TC(M) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12)
#define MAPDEC_FOR_N(M) M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12)
