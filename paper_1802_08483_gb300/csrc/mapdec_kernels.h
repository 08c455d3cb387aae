// Host-side declarations of the kernel launchers (internal to libmapdec.so).
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mapdec_dev.cuh"

namespace mdk {

// Raise a kernel's dynamic shared-memory opt-in to the device's per-block
// maximum less the kernel's static shared memory, once per device: the
// attribute is held per device, so a process that launches on several GPUs
// sets it on each.  `done` has one bit per device (devices 0..63; beyond that
// the attribute is set on every call).  Safe to call from several threads:
// concurrent first calls may both set the same value, which is harmless.
template <typename Kern>
cudaError_t smem_optin_once(Kern kern, std::atomic<uint64_t> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

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
// Tensor-core forward producer (producers_tc.cuh): which frames it serves,
// its shared memory, and its launch.
bool fwd_tc_supported(int q, int n, int I);
size_t fwd_tc_smem_bytes(const FrameDev &f);
// The priors of a frame split into bf16 pieces in the tensor-core operand
// layout (k_prior_split): 8-row groups allocated, bytes, and the launch (one
// thread per group, 8-column chunk and row; max_threads = the largest frame's).
inline int prior_split_groups(const FrameDev &f) { return (f.N + 16 + 7) / 8; }
size_t prior_split_bytes(const FrameDev &f);
cudaError_t launch_prior_split(const FrameDev *frames, int nframes, long long max_threads,
                               cudaStream_t st);
cudaError_t launch_fwd_tc(int n, int I, const FrameDev *frames, const Work *work, int nwork,
                          size_t smem, cudaStream_t st);
// Per-symbol-codebook producers (producers_ps.cuh): any (n, I) the lattices
// support, q <= 256; work items (frame, symbol * psT + chunk).
cudaError_t launch_fwd_ps(int n, int I, const FrameDev *frames, const Work *work, int nwork,
                          cudaStream_t st);
cudaError_t launch_bwd_ps(int n, int I, bool grad, const FrameDev *frames, const Work *work,
                          int nwork, size_t smem, cudaStream_t st);
size_t bwd_ps_smem_bytes(const FrameDev &f, bool grad);
int ps_chunk_states(int q, int M);  // start states per work item
// Tensor-core APP producer (decode mode): same class rule, S2 <= 128.
size_t bwd_tc_smem_bytes(const FrameDev &f);
cudaError_t launch_bwd_tc(int n, int I, const FrameDev *frames, const Work *work, int nwork,
                          size_t smem, cudaStream_t st);
constexpr size_t kTcMinSmem = 80 * 1024;  // caps the tensor-core producers at 2 CTAs per SM
constexpr int kTcChunkCols = 80;          // A-operand columns per chunk of the APP producer
size_t bwd_smem_bytes(const FrameDev &f, bool grad);

// dst[k] = src[k] for n16 16-byte words (both 16-byte aligned device addresses,
// either of them the device mapping of pinned host memory), by the SMs.
cudaError_t launch_copy16(void *dst, const void *src, size_t n16, int sms, cudaStream_t st);
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
                                        int nwork, size_t smem, cudaStream_t st);            \
    cudaError_t launch_fwd_tc_I##IB(int n, const FrameDev *frames, const Work *work,         \
                                    int nwork, size_t smem, cudaStream_t st);                \
    cudaError_t launch_bwd_tc_I##IB(int n, const FrameDev *frames, const Work *work,         \
                                    int nwork, size_t smem, cudaStream_t st);                \
    cudaError_t launch_fwd_ps_I##IB(int n, const FrameDev *frames, const Work *work,         \
                                    int nwork, cudaStream_t st);                             \
    cudaError_t launch_bwd_ps_I##IB##_plain(int n, const FrameDev *frames, const Work *work, \
                                            int nwork, size_t smem, cudaStream_t st);        \
    cudaError_t launch_bwd_ps_I##IB##_grad(int n, const FrameDev *frames, const Work *work,  \
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
