// Host-side declarations of the kernel launchers (internal to libmapdec.so).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mapdec_dev.cuh"

namespace mdk {

// Producers dispatched on (n, I); pairs without a compiled specialisation run
// the run-time lattice.  smem = dynamic shared bytes (see *_smem_bytes).
cudaError_t launch_fwd(int n, int I, const FrameDev *frames, const Work *work, int nwork,
                       size_t smem, cudaStream_t st);
cudaError_t launch_bwd(int n, int I, bool grad, const FrameDev *frames, const Work *work,
                       int nwork, size_t smem, cudaStream_t st);
cudaError_t launch_rmetric(int n, int I, const FrameDev *frame, long long nthreads,
                           cudaStream_t st);
bool specialised(int n, int I);
size_t fwd_smem_bytes(const FrameDev &f);
size_t bwd_smem_bytes(const FrameDev &f, bool grad);

cudaError_t launch_pack(const FrameDev *frames, const uint8_t *const *rx_bytes,
                        uint32_t *const *rx_words, int nframes, long long max_words,
                        cudaStream_t st);
size_t chain_smem_bytes(const FrameDev &f);
// threads: 128, 256 or 512 (anything else selects the default, 256)
cudaError_t launch_chain(const FrameDev *frames, const Work *work, int nwork, size_t smem,
                         int threads, cudaStream_t st);
cudaError_t launch_finalize(const FrameDev *frames, const Work *work, int nwork, int nframes,
                            int grad, cudaStream_t st, bool reduce = true);
size_t chain_state_bytes();
int finalize_chunks(int N);  // work items (frame, chunk) per frame

// per-I launchers defined in producers_i<I>.cu
#define MAPDEC_DECLARE_I(IB)                                                                 \
    cudaError_t launch_fwd_I##IB(int n, const FrameDev *frames, const Work *work, int nwork, \
                                 size_t smem, cudaStream_t st);                               \
    cudaError_t launch_bwd_I##IB(int n, bool grad, const FrameDev *frames, const Work *work, \
                                 int nwork, size_t smem, cudaStream_t st);                    \
    cudaError_t launch_rmetric_I##IB(int n, const FrameDev *frame, long long nthreads,       \
                                     cudaStream_t st);                                        \
    cudaError_t launch_bwd_I##IB##_plain(int n, const FrameDev *frames, const Work *work,    \
                                         int nwork, size_t smem, cudaStream_t st);            \
    cudaError_t launch_bwd_I##IB##_grad(int n, const FrameDev *frames, const Work *work,     \
                                        int nwork, size_t smem, cudaStream_t st);
MAPDEC_DECLARE_I(1)
MAPDEC_DECLARE_I(2)
MAPDEC_DECLARE_I(3)
cudaError_t launch_fwd_rt(const FrameDev *frames, const Work *work, int nwork, size_t smem,
                          cudaStream_t st);
cudaError_t launch_bwd_rt(bool grad, const FrameDev *frames, const Work *work, int nwork,
                          size_t smem, cudaStream_t st);
cudaError_t launch_rmetric_rt(const FrameDev *frame, long long nthreads, cudaStream_t st);

constexpr int kMaxSpecN = 12;  // n = 1..12 specialised for I = 1, 2, 3

}  // namespace mdk
