// Host side of libmapdec.so: argument validation, tile planning, device
// memory, launch sequencing (optionally captured in a CUDA graph) and the
// C ABI declared in include/mapdec.h.
//
// Launch sequence of one run (per wave of frames that fit the scratch budget):
//   pack rx bits -> forward producers (lattice + W, per (n, I) class)
//   -> forward and backward chains (one CTA per frame and direction)
//   -> backward producers (lattice + APP / tangent partial sums)
//   -> finalize (APPs, d logP / d prior, FP64 gradient reduction)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mapdec.h"
#include "mapdec_kernels.h"

using namespace mdk;

namespace {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
struct CudaErr {
    cudaError_t e;
};
// MAPDEC_VERBOSE=1 (read once) names the failing CUDA call on stderr; the
// caller always gets the MAPDEC_* status.
bool verbose() {
    static const bool v = [] {
        const char *e = std::getenv("MAPDEC_VERBOSE");
        return e && std::atoi(e) != 0;
    }();
    return v;
}
#define CK(x)                                                                            \
    do {                                                                                 \
        cudaError_t _e = (x);                                                            \
        if (_e != cudaSuccess) {                                                         \
            if (verbose())                                                               \
                std::fprintf(stderr, "libmapdec: %s (%s:%d): %s\n", cudaGetErrorName(_e), \
                             __FILE__, __LINE__, #x);                                    \
            throw CudaErr{_e};                                                           \
        }                                                                                \
    } while (0)

int map_cuda(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return MAPDEC_ERR_NOMEM;
    return MAPDEC_ERR_CUDA;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of pinned (page-locked, mapped) host memory, or null for
// pageable host memory and for device memory.
void *mapped_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int device_sms() {
    static std::atomic<int> cache[64];  // 0 = not yet read on that device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

// Host <-> device copies of the batch's inputs and outputs.  Pinned host
// memory is moved by the SMs through its device mapping: a copy engine's
// first pass over a buffer that kernels have just written or read runs at a
// small fraction of its rate (measured: 14 against 210 GB/s on the 0.8 GB
// prior and APP buffers right after a decode), while the SM copy is not
// affected.  Small copies (latency-bound either way), unaligned and pageable
// host buffers go through the copy engine.
constexpr size_t kSmCopyMin = 1 << 20;
bool sm_copy(const void *a, const void *b, size_t bytes) {
    return bytes >= kSmCopyMin && (((uintptr_t)a | (uintptr_t)b) & 15u) == 0;
}
void copy_in(void *dst_dev, const void *src, size_t bytes, cudaStream_t st) {
    if (bytes == 0 || src == dst_dev) return;  // already resident (caller passed the batch's own buffer)
    if (is_device_ptr(src)) {
        CK(cudaMemcpyAsync(dst_dev, src, bytes, cudaMemcpyDeviceToDevice, st));
        return;
    }
    void *m = mapped_host(src);
    if (m && sm_copy(m, dst_dev, bytes)) {
        // the tail (under 16 bytes) by the copy engine from the host address
        const size_t head = bytes / 16 * 16;
        CK(launch_copy16(dst_dev, m, bytes / 16, device_sms(), st));
        if (head < bytes)
            CK(cudaMemcpyAsync(static_cast<char *>(dst_dev) + head,
                               static_cast<const char *>(src) + head, bytes - head,
                               cudaMemcpyHostToDevice, st));
        return;
    }
    CK(cudaMemcpyAsync(dst_dev, src, bytes, cudaMemcpyHostToDevice, st));
}
void copy_out(void *dst, const void *src_dev, size_t bytes, cudaStream_t st) {
    if (bytes == 0 || !dst || dst == src_dev) return;
    if (is_device_ptr(dst)) {
        CK(cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDeviceToDevice, st));
        return;
    }
    void *m = mapped_host(dst);
    if (m && sm_copy(m, src_dev, bytes)) {
        const size_t head = bytes / 16 * 16;
        CK(launch_copy16(m, src_dev, bytes / 16, device_sms(), st));
        if (head < bytes)
            CK(cudaMemcpyAsync(static_cast<char *>(dst) + head,
                               static_cast<const char *>(src_dev) + head, bytes - head,
                               cudaMemcpyDeviceToHost, st));
        return;
    }
    CK(cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDeviceToHost, st));
}

size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Validate one frame description; returns a MAPDEC_* status.
int validate(int q, int n, int N, double Pi, double Pd, double Ps, int I, int xmax) {
    if (q < 2 || n < 1 || n > 31 || N < 1 || I < 1 || I > kMaxI || xmax < 0) return MAPDEC_ERR_ARG;
    if ((long long)q > (1ll << n)) return MAPDEC_ERR_ARG;
    if (n * (I + 1) + 1 > kMaxMN) return MAPDEC_ERR_UNSUPPORTED;
    if (!(Pi >= 0 && Pd >= 0 && Ps >= 0 && Ps <= 1 && Pi + Pd < 1)) return MAPDEC_ERR_ARG;
    if (!std::isfinite(Pi) || !std::isfinite(Pd) || !std::isfinite(Ps)) return MAPDEC_ERR_ARG;
    if ((long long)xmax > (1ll << 24)) return MAPDEC_ERR_UNSUPPORTED;
    return MAPDEC_OK;
}

// Codebook (q*n bytes, host or device) -> packed words; checks bits and distinctness.
int pack_codebook(const uint8_t *cb, int q, int n, std::vector<uint32_t> &out) {
    if (!cb) return MAPDEC_ERR_ARG;
    std::vector<uint8_t> h((size_t)q * n);
    if (is_device_ptr(cb)) {
        if (cudaMemcpy(h.data(), cb, h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
            return MAPDEC_ERR_CUDA;
    } else {
        std::memcpy(h.data(), cb, h.size());
    }
    out.assign(q, 0u);
    std::set<uint32_t> seen;
    for (int d = 0; d < q; ++d) {
        uint32_t w = 0;
        for (int r = 0; r < n; ++r) {
            const uint8_t b = h[(size_t)d * n + r];
            if (b > 1) return MAPDEC_ERR_ARG;
            if (b) w |= (1u << r);
        }
        if (!seen.insert(w).second) return MAPDEC_ERR_ARG;  // encoding must be injective
        out[d] = w;
    }
    return MAPDEC_OK;
}

// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------
constexpr int kPhases = 5;  // pack, forward producers, chains, backward producers, finalize
constexpr int kRegions = 3; // rotating scratch regions when frames need several waves
constexpr size_t kFwdSmemBudget = 110 * 1024;
constexpr size_t kBwdSmemBudget = 110 * 1024;  // two CTAs per SM
constexpr size_t kChainSmemBudget = 100 * 1024;  // two chains per SM
constexpr int kChainStages = 2;

struct FrameHost {
    mapdec_frame_desc_t d;
    std::vector<uint32_t> cw;
    int64_t rx_off = 0;     // byte offset in the concatenated rx buffer
    int64_t sym_off = 0;    // row offset (rows of q floats) in priors / APP buffers
    int64_t rxw_off = 0;    // word offset in the packed rx buffer
    int64_t cw_off = 0;     // word offset in the packed codebook buffer
    FrameDev dev{};         // shape, constants; pointers filled per wave
    size_t scratch_floats = 0;
    double cost = 0.0;
    int segK = 0, nseg = 1; // segmented mode: symbols per segment, segments
    bool store = false;     // keep the receiver metrics in HBM for the APP producer
    bool tc = false;        // forward producer on the tensor cores
    bool tcb = false;       // APP producer on the tensor cores
    std::vector<float> phi0, phiN;  // boundary drift priors (stream decoding), or empty
    int64_t phi_off = 0;    // float offset of phi0 (then phiN) in the batch's buffer
};

// Stored receiver metrics of a frame: T tiles of P*MN rows x roundup4(q) floats.
size_t metric_store_floats(const FrameDev &f) {
    return (size_t)f.T * f.P * f.MN * (size_t)((f.q + 3) & ~3);
}

// Tuning table: launch parameters per (q, n, I) class, set through
// mapdec_tune_set (normally from a tuner's measurements).  Read when a batch
// is planned.
struct TuneEntry {
    int q, n, I;
    mapdec_tune_t t;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;

bool tune_lookup(int q, int n, int I, mapdec_tune_t &out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto &e : g_tune)
        if (e.q == q && e.n == n && e.I == I) {
            out = e.t;
            return true;
        }
    return false;
}

// Fill shape-dependent fields of dev (P, S, T, nsub, ...) for received length rho.
// tune (may be null) holds the class's tuned parameters (0 = planner's choice);
// forceP > 0 (testing) overrides the tile size.
void plan_shape(FrameDev &f, const mapdec_frame_desc_t &d, bool grad, int forceP,
                const mapdec_tune_t *tune = nullptr) {
    f.q = d.q; f.n = d.n; f.N = d.N; f.I = d.I; f.xmax = d.xmax;
    f.M = 2 * d.xmax + 1;
    f.Mp = (int)rup(f.M, 4);
    f.MN = d.n * (d.I + 1) + 1;
    f.MNS = (f.MN & 1) ? f.MN : f.MN + 1;
    f.rho = d.rx_len;
    f.wblk = (long long)rup((size_t)f.M * f.MNS, 4);
    const double Pt = 1.0 - d.Pi - d.Pd;
    const double kappa = 2.0;        // weight per received bit (see FrameDev)
    const double w1 = kappa * 0.5 * d.Pi;
    double wp = 1.0;
    for (int a = 0; a <= kMaxI; ++a) {
        f.wpow[a] = (a <= d.I) ? (float)wp : 0.f;
        f.wder[a] = (a >= 1 && a <= d.I) ? (float)(a * std::pow(w1, a - 1)) : 0.f;
        wp *= w1;
    }
    f.Pd = (float)d.Pd;
    f.qsame = (float)(kappa * Pt * (1.0 - d.Ps));
    f.qdiff = (float)(kappa * Pt * d.Ps);
    f.dPi = d.Pi; f.dPd = d.Pd; f.dPs = d.Ps; f.dPt = Pt;
    f.kappa = kappa;
    f.logk = std::log(kappa);
    f.seg_i0 = 0;
    f.seg_i1 = d.N;
    f.fin_base = 0;
    f.fin_total = finalize_chunks(d.N);
    f.chain_flags = 0;
    // bounded waits: a recursion gives up on a copy after this many polls
    f.wait_limit = 1u << 26;
    f.test_flags = 0;
    if (const char *e = std::getenv("MAPDEC_TEST_STALL_CHAIN")) {  // testing: the timeout path
        if (std::atoi(e) == 1) {
            f.test_flags |= TEST_SKIP_FIRST_COPY;
            f.wait_limit = 4096;
        }
    }
    f.ckpt = nullptr;
    f.bedge = nullptr;
    f.cst = nullptr;

    auto symbols_span = [&](long long Ppos) -> int {
        return (int)((Ppos - 1 + 2LL * d.xmax) / d.n + 2);
    };
    // positions per sub-tile
    static const int cand[] = {64, 48, 32, 24, 16, 12, 8, 6, 4, 2, 1};
    const int want = forceP > 0 ? forceP : (tune && tune->P > 0 ? tune->P : 0);
    int P = 1;
    for (int pass = want > 0 ? 0 : 1; pass < 2; ++pass)
    for (int c : cand) {
        if (pass == 0 && c != want) continue;
        FrameDev t = f;
        t.P = t.Pf = c;
        t.S = t.Sf = symbols_span(c);
        t.nsub = std::max(1, 256 / c);
        t.S2 = symbols_span((long long)c * t.nsub);
        if (fwd_smem_bytes(t) > kFwdSmemBudget) continue;
        while (t.nsub > 1 && bwd_smem_bytes(t, grad) > kBwdSmemBudget) {
            t.nsub /= 2;
            t.S2 = symbols_span((long long)c * t.nsub);
        }
        if (bwd_smem_bytes(t, grad) > kBwdSmemBudget) continue;
        P = c;
        pass = 2;  // found: leave both loops
        break;
    }
    f.P = P;
    f.S = symbols_span(P);
    f.nsub = std::max(1, 256 / P);
    f.S2 = symbols_span((long long)P * f.nsub);
    while (f.nsub > 1 && bwd_smem_bytes(f, grad) > kBwdSmemBudget) {
        f.nsub /= 2;
        f.S2 = symbols_span((long long)P * f.nsub);
    }
    if (tune && tune->nsub > 0 && tune->nsub <= f.nsub) {
        f.nsub = tune->nsub;
        f.S2 = symbols_span((long long)P * f.nsub);
    }
    if (const char *e = std::getenv("MAPDEC_FORCE_NSUB")) {  // testing override
        const int ns = std::atoi(e);
        if (ns >= 1 && ns <= f.nsub) {
            f.nsub = ns;
            f.S2 = symbols_span((long long)P * f.nsub);
        }
    }
    f.T = (int)((f.rho + 1 + P - 1) / P);
    f.T2 = (f.T + f.nsub - 1) / f.nsub;
    f.Pf = f.P;
    f.Sf = f.S;
    f.Tf = f.T;
    // chain chunk: all states at once if it fits, else the largest power of two;
    // as many stages in flight as the budget allows (at least two)
    size_t cbud = kChainSmemBudget;
    if (tune && tune->chain_budget_kb >= 16 && tune->chain_budget_kb <= 220)
        cbud = (size_t)tune->chain_budget_kb * 1024;
    if (const char *e = std::getenv("MAPDEC_CHAIN_BUDGET_KB")) {  // tuning override
        const int kb = std::atoi(e);
        if (kb >= 16 && kb <= 220) cbud = (size_t)kb * 1024;
    }
    int stages = kChainStages;
    if (tune && tune->chain_stages >= 2 && tune->chain_stages <= 8) stages = tune->chain_stages;
    if (const char *e = std::getenv("MAPDEC_CHAIN_STAGES")) {  // tuning override
        const int v = std::atoi(e);
        if (v >= 2 && v <= 8) stages = v;
    }
    auto chain_fits = [&](int cd, int stg) {
        FrameDev t = f;
        t.chainCD = cd;
        t.chainStages = stg;
        return chain_smem_bytes(t) <= cbud;
    };
    // the fewest chunks per step that fit, equal in size (at most 64 chunks)
    int CD = f.M;
    for (int nck = 1; nck <= 64; ++nck) {
        CD = (f.M + nck - 1) / nck;
        if (chain_fits(CD, stages)) break;
    }
    if (const char *e = std::getenv("MAPDEC_CHAIN_CD")) {  // tuning / testing override
        const int cd = std::atoi(e);
        if (cd >= 32) {
            FrameDev t = f;
            t.chainCD = std::min(cd, f.M);
            t.chainStages = stages;
            if (chain_smem_bytes(t) <= 227 * 1024) CD = t.chainCD;
        }
    }
    // at most 64 chunks per step (the chain's chunk table)
    CD = std::max(CD, (f.M + 63) / 64);
    f.chainCD = CD;
    f.chainStages = stages;
}

// Forward tile of the tensor-core producer: up to two lattices per thread
// (Pf <= 512 / q positions), at most 256 symbols from the 8-aligned first one
// (the MMA's N), the shared memory within the two-CTA budget: frames with wide
// drift limits get short tiles (their priors block is large), narrow ones long
// tiles; among those, the tile that keeps the most threads busy in its rounds
// of lattices.  Sets Pf, Sf, Tf; false if no tile fits (the CUDA-core producer
// is used).
bool plan_fwd_tc(FrameDev &f) {
    if (!fwd_tc_supported(f.q, f.n, f.I)) return false;
    // among the tiles that fit, the most positions per round of lattices
    // (P / ceil(P q / 256): one lattice per thread and round), then the longest
    int best = 0;
    double best_score = 0.0;
    for (int P = std::max(1, 512 / f.q); P >= 1; --P) {
        FrameDev t = f;
        t.Pf = P;
        t.Sf = (int)std::min<long long>(((long long)P - 1 + 2LL * f.xmax) / f.n + 2, f.N);
        if (((t.Sf + 7 + 15) & ~15) > 256) continue;
        if (fwd_tc_smem_bytes(t) > kFwdSmemBudget) continue;
        const double score = (double)P / (double)((P * f.q + kThreads - 1) / kThreads);
        if (score > best_score) {
            best_score = score;
            best = P;
        }
    }
    if (best == 0) return false;
    f.Pf = best;
    f.Sf = (int)std::min<long long>(((long long)best - 1 + 2LL * f.xmax) / f.n + 2, f.N);
    f.Tf = (int)((f.rho + 1 + best - 1) / best);
    return true;
}

// APP-producer tiling of the tensor-core kernel (decode mode): one lattice per
// thread per sub-tile (P = 256 / q positions), as many sub-tiles per super-tile
// (up to 256 positions) as keep its symbols within the 128 accumulator rows,
// shared memory within the two-CTA budget.  Sets P, S, nsub, S2, T, T2; false
// if no tiling fits (the CUDA-core producer and the planner's tiling stay).
bool plan_bwd_tc(FrameDev &f) {
    if (!fwd_tc_supported(f.q, f.n, f.I)) return false;
    auto span = [&](long long Ppos) -> int {
        return (int)std::min<long long>((Ppos - 1 + 2LL * f.xmax) / f.n + 2, f.N);
    };
    for (int P = 256 / f.q; P >= 1; --P) {
        FrameDev t = f;
        t.P = P;
        t.S = span(P);
        int nsub = std::max(1, 256 / P);
        while (nsub > 1 && span((long long)P * nsub) > 128) --nsub;
        t.nsub = nsub;
        t.S2 = span((long long)P * nsub);
        if (t.S2 > 128 || bwd_tc_smem_bytes(t) > kBwdSmemBudget) continue;
        t.T = (int)((t.rho + 1 + P - 1) / P);
        t.T2 = (t.T + t.nsub - 1) / t.nsub;
        f = t;
        return true;
    }
    return false;
}

size_t frame_scratch_floats(const FrameDev &f, bool grad) {
    size_t s = 0;
    if (f.Pgroups) s += rup(prior_split_bytes(f) / 4, 64);  // priors split for the tensor cores
    s += rup((size_t)f.N * f.wblk + 16, 64);             // W (+ tail slack for bulk copies)
    s += rup((size_t)(f.N + 1) * f.Mp, 64) * 2;          // alpha, beta
    s += rup((size_t)f.T2 * f.S2 * f.q, 64);             // Lp
    if (grad) s += rup((size_t)f.T2 * f.S2 * 3, 64);     // Gp
    s += 3 * rup((size_t)(f.N + 1) * 2, 64);             // thf, mcf, thb (doubles)
    if (grad) s += rup((size_t)finalize_chunks(f.N) * 3 * 2, 64);  // Gc (doubles)
    return s;
}

// Segmented mode: W, alpha, beta and the APP partials for one segment of K
// symbols, plus forward checkpoints every K symbols.
int seg_supertiles(const FrameDev &f, int K) {
    const long long P2 = (long long)f.P * f.nsub;
    return (int)(((long long)f.n * K + 2LL * f.xmax) / P2 + 3);
}
size_t frame_scratch_floats_seg(const FrameDev &f, int K, int S, bool grad) {
    const int T2s = seg_supertiles(f, K);
    const int cps = finalize_chunks(K);
    size_t s = 0;
    if (f.Pgroups) s += rup(prior_split_bytes(f) / 4, 64);  // priors split for the tensor cores
    s += 2 * rup((size_t)K * f.wblk + 16, 64);           // W of a segment, two buffers
    s += 4 * rup((size_t)(K + 1) * f.Mp, 64);            // alpha, beta rows of a segment, two buffers
    s += rup((size_t)T2s * f.S2 * f.q, 64);              // Lp of one segment
    if (grad) s += rup((size_t)T2s * f.S2 * 3, 64);      // Gp
    s += 3 * rup((size_t)(f.N + 1) * 2, 64);             // thf, mcf, thb
    if (grad) s += rup((size_t)S * cps * 3 * 2, 64);     // Gc
    s += rup((size_t)(S + 1) * f.Mp, 64);                // forward checkpoints
    s += rup((size_t)f.Mp, 64);                          // backward boundary row
    s += rup(2 * chain_state_bytes() / 4 + 1, 64);       // chain states
    return s;
}

double frame_cost(const FrameDev &f) {
    // algorithmic flop estimate used for load balancing and reporting
    const double cells = (f.I + 1) * f.n * (f.n + 1) / 2.0 + (f.n + 1);
    const double lat = (double)(f.rho + 1) * f.q * cells * (2.0 * f.I + 3.0);
    const double band = (double)f.N * f.M * f.MN;
    return 2.0 * lat + 4.0 * band * f.q + 4.0 * band;
}

// Producer launches are grouped by (n, I) (the compiled lattice) and by the
// forward producer's kind.
using ClassKey = std::tuple<int, int, int>;  // n, I, tensor-core bits (kTcFwd | kTcBwd)

constexpr int kTcFwd = 1, kTcBwd = 2;  // ClassKey / FrameHost tensor-core bits
constexpr int kTcMinSymbols = 36;      // default rule: tensor-core forward producer from this
                                       // many symbols per tile
constexpr int kPerSym = 4;             // ClassKey: per-symbol-codebook producers

struct ClassLaunch {
    int n, I;
    bool tc = false;   // forward producer on the tensor cores (producers_tc.cuh)
    bool tcb = false;  // APP producer on the tensor cores
    bool ps = false;   // per-symbol-codebook producers (producers_ps.cuh)
    Work *d_fwd = nullptr; int nfwd = 0; size_t smem_fwd = 0;
    Work *d_bwd = nullptr; int nbwd = 0; size_t smem_bwd = 0;
};

// One segment index of a segmented wave: descriptors and work lists.
struct SegLaunch {
    FrameDev *d_frames = nullptr;
    std::vector<ClassLaunch> cls;
    Work *d_rec = nullptr; int nrec = 0;    // forward chains (record)
    Work *d_bw = nullptr; int nbw = 0;      // forward replay + backward chains
    Work *d_fin = nullptr; int nfin = 0;
    int nframes = 0;
    // order between the producer stream and the recursion stream
    cudaEvent_t ev_fwd = nullptr, ev_rec = nullptr;             // recording sweep
    cudaEvent_t ev_fwd2 = nullptr, ev_chain2 = nullptr, ev_bwd = nullptr;  // recompute sweep
};

struct Wave {
    int f0 = 0, f1 = 0;
    std::vector<SegLaunch> segs;  // segmented mode
    FrameDev *d_frames = nullptr;
    std::vector<ClassLaunch> cls;
    Work *d_chain = nullptr; int nchain = 0; size_t smem_chain = 0;
    Work *d_fin = nullptr; int nfin = 0;
    const uint8_t **d_rxptr = nullptr;
    uint32_t **d_rxwptr = nullptr;
    long long max_words = 0;
    long long prior_split_threads = 0;  // the largest tensor-core frame's k_prior_split work
};

}  // namespace

// ---------------------------------------------------------------------------
// batch object
// ---------------------------------------------------------------------------
struct mapdec_batch {
    int nframes = 0;
    int flags = 0;
    bool grad = false;
    std::vector<FrameHost> fr;
    int64_t rx_total = 0, prior_total = 0, rxw_total = 0, cw_total = 0;
    uint8_t *d_rx = nullptr;
    float *d_priors = nullptr;
    float *d_app = nullptr;
    float *d_dpriors = nullptr;
    float *d_ext = nullptr;
    double *d_loglik = nullptr;
    double *d_dchan = nullptr;
    int *d_status = nullptr;
    uint32_t *d_rxw = nullptr;
    uint32_t *d_cw = nullptr;
    float *d_phi = nullptr;       // boundary drift priors of the frames that have them
    int64_t phi_total = 0;
    float *d_scratch = nullptr;
    size_t scratch_floats = 0;   // largest wave's scratch
    size_t region_floats = 0;    // stride between rotating scratch regions
    int regions = 1;
    cudaStream_t aux_stream = nullptr;  // chains run here, overlapping the producers
    std::vector<cudaEvent_t> dep;       // per wave: forward done, chains done
    std::vector<Wave> waves;
    std::vector<void *> allocs;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
    cudaGraphExec_t gexec = nullptr;
    bool graph_grad = false;
    int64_t last_launches = 0;
    int64_t launches_per_run[2] = {0, 0};
    bool timing = false;
    bool segmented = false;
    int chain_threads = 0;  // 0: the chain kernel's default

    std::vector<cudaEvent_t> events;  // per wave and phase: begin, end
    std::vector<cudaEvent_t> seg_events;  // segmented runs: ordering events of every segment

    void *dalloc(size_t bytes) {
        void *p = nullptr;
        CK(cudaMalloc(&p, std::max<size_t>(bytes, 16)));
        allocs.push_back(p);
        return p;
    }
    ~mapdec_batch() {
        if (gexec) cudaGraphExecDestroy(gexec);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        for (cudaEvent_t e : seg_events) cudaEventDestroy(e);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (aux_stream) cudaStreamDestroy(aux_stream);
        for (cudaEvent_t e : dep) cudaEventDestroy(e);

        for (void *p : allocs) cudaFree(p);
    }
};

// Single-frame handle.  Its batches of one frame are planned and allocated
// once for the largest admissible received length rho_max = tau + xmax; a call
// with any rho in [tau - xmax, tau + xmax] only rewrites the frame descriptor
// and the producers' work counts (the work lists are prefixes of rho_max's).
struct mapdec {
    int q, n, N, I, xmax;
    double Pi, Pd, Ps;
    std::vector<uint8_t> codebook;  // host copy
    cudaStream_t stream = nullptr;
    int64_t rho_max = 0;
    mapdec_batch *b = nullptr;      // decode (APPs, extrinsic outputs), made by mapdec_create
    mapdec_batch *bg = nullptr;     // gradient mode, made by the first mapdec_loglik_grad
    float *d_rout = nullptr;        // receiver-metric dump, (rho_max+1)*q*MN floats, first use
    float *d_phi = nullptr;         // boundary drift priors: start, end (2 M floats), at create
    bool use_phi0 = false, use_phiN = false;
    ~mapdec() {
        delete b;
        delete bg;
        if (d_rout) cudaFree(d_rout);
        if (d_phi) cudaFree(d_phi);
    }
};

namespace {

// Segmented mode: per segment index, one descriptor per frame (bounds and
// buffer bases shifted so that absolute symbol, row and super-tile indices land
// in the frame's one-segment buffers) and the work lists of that segment.
void build_segments(mapdec_batch *b, Wave &w, const std::vector<FrameDev> &devs,
                    const std::map<ClassKey, std::vector<int>> &byclass) {
    const int nw = w.f1 - w.f0;
    int Smax = 0;
    for (int k = 0; k < nw; ++k) Smax = std::max(Smax, b->fr[w.f0 + k].nseg);
    w.segs.resize(Smax);
    for (int s = 0; s < Smax; ++s) {
        SegLaunch &sl = w.segs[s];
        std::vector<FrameDev> sd(devs);
        std::vector<Work> rec, bw, fin;
        for (int k = 0; k < nw; ++k) {
            const FrameHost &h = b->fr[w.f0 + k];
            if (s >= h.nseg) continue;
            FrameDev f = devs[k];
            const int K = h.segK, i0 = s * K, i1 = std::min(f.N, i0 + K);
            const long long P2 = (long long)f.P * f.nsub;
            const long long plo = std::max(0LL, (long long)f.n * i0 - f.xmax);
            const long long t2first = plo / P2;
            auto shift = [](void *p, long long bytes) {
                return (void *)((char *)p - bytes);
            };
            f.seg_i0 = i0;
            f.seg_i1 = i1;
            const size_t wst = rup((size_t)K * f.wblk + 16, 64), ast = rup((size_t)(K + 1) * f.Mp, 64);
            const size_t buf = (size_t)(s & 1);
            f.W = (float *)shift(devs[k].W + buf * wst, (long long)i0 * f.wblk * 4);
            f.alpha = (float *)shift(devs[k].alpha + buf * ast, (long long)i0 * f.Mp * 4);
            f.beta = (float *)shift(devs[k].beta + buf * ast, (long long)i0 * f.Mp * 4);
            f.Lp = (float *)shift(devs[k].Lp, t2first * f.S2 * f.q * 4);
            if (devs[k].Gp) f.Gp = (float *)shift(devs[k].Gp, t2first * f.S2 * 3 * 4);
            f.ckpt = devs[k].ckpt + (size_t)s * f.Mp;
            f.fin_base = s * finalize_chunks(K);
            sd[k] = f;
            rec.push_back({k, 0});
            bw.push_back({k, 2});
            bw.push_back({k, 1});
            for (int c = 0; c < finalize_chunks(i1 - i0); ++c) fin.push_back({k, f.fin_base + c});
        }
        sl.nframes = nw;
        sl.d_frames = (FrameDev *)b->dalloc(sizeof(FrameDev) * nw);
        CK(cudaMemcpy(sl.d_frames, sd.data(), sizeof(FrameDev) * nw, cudaMemcpyHostToDevice));
        auto upload = [&](const std::vector<Work> &v, Work *&dst, int &cnt) {
            cnt = (int)v.size();
            dst = (Work *)b->dalloc(sizeof(Work) * std::max<size_t>(v.size(), 1));
            if (!v.empty())
                CK(cudaMemcpy(dst, v.data(), sizeof(Work) * v.size(), cudaMemcpyHostToDevice));
        };
        for (cudaEvent_t *e : {&sl.ev_fwd, &sl.ev_rec, &sl.ev_fwd2, &sl.ev_chain2, &sl.ev_bwd}) {
            CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
            b->seg_events.push_back(*e);
        }
        upload(rec, sl.d_rec, sl.nrec);
        upload(bw, sl.d_bw, sl.nbw);
        upload(fin, sl.d_fin, sl.nfin);
        for (const auto &kv : byclass) {
            ClassLaunch c;
            c.n = std::get<0>(kv.first);
            c.I = std::get<1>(kv.first);
            c.tc = (std::get<2>(kv.first) & kTcFwd) != 0;
            c.tcb = (std::get<2>(kv.first) & kTcBwd) != 0;
            c.ps = (std::get<2>(kv.first) & kPerSym) != 0;
            std::vector<Work> fw, bwk;
            for (int k : kv.second) {
                const FrameHost &h = b->fr[w.f0 + k];
                if (s >= h.nseg) continue;
                const FrameDev &f = sd[k];
                const long long P2 = (long long)f.P * f.nsub;
                const long long plo = std::max(0LL, (long long)f.n * f.seg_i0 - f.xmax);
                const long long phi = std::min(f.rho, (long long)f.n * (f.seg_i1 - 1) + f.xmax);
                for (long long t = plo / f.Pf; t <= phi / f.Pf; ++t) fw.push_back({k, (int)t});
                for (long long t = plo / P2; t <= phi / P2; ++t) bwk.push_back({k, (int)t});
                c.smem_fwd = std::max(c.smem_fwd, c.tc ? fwd_tc_smem_bytes(f) : fwd_smem_bytes(f));
                c.smem_bwd = std::max(c.smem_bwd, c.ps    ? bwd_ps_smem_bytes(f, b->grad)
                                                  : c.tcb ? bwd_tc_smem_bytes(f)
                                                          : bwd_smem_bytes(f, b->grad));
            }
            upload(fw, c.d_fwd, c.nfwd);
            upload(bwk, c.d_bwd, c.nbwd);
            sl.cls.push_back(c);
        }
    }
}

// Build the batch: plan, allocate, upload descriptors.  Throws CudaErr.
int build_batch(mapdec_batch *b, const mapdec_frame_desc_t *frames, int nf, int flags,
                int64_t budget, int forceP) {
    b->nframes = nf;
    b->flags = flags;
    b->grad = (flags & MAPDEC_BATCH_GRAD) != 0;
    b->fr.resize(nf);
    for (int i = 0; i < nf; ++i) {
        FrameHost &h = b->fr[i];
        h.d = frames[i];
        int st = validate(h.d.q, h.d.n, h.d.N, h.d.Pi, h.d.Pd, h.d.Ps, h.d.I, h.d.xmax);
        if (st) return st;
        const long long tau = (long long)h.d.n * h.d.N;
        if (h.d.rx_len < 0) return MAPDEC_ERR_ARG;
        if (std::llabs(h.d.rx_len - tau) > h.d.xmax) return MAPDEC_ERR_DRIFT_RANGE;
        {
            // boundary drift priors (stream decoding): host or device, copied here
            const int M = 2 * h.d.xmax + 1;
            auto read_prior = [&](const float *src, std::vector<float> &dst) -> int {
                if (!src) return MAPDEC_OK;
                dst.resize(M);
                if (is_device_ptr(src)) {
                    CK(cudaMemcpy(dst.data(), src, (size_t)M * 4, cudaMemcpyDeviceToHost));
                } else {
                    std::memcpy(dst.data(), src, (size_t)M * 4);
                }
                double tot = 0.0;
                for (float v : dst) {
                    if (!(v >= 0.f) || !std::isfinite(v)) return MAPDEC_ERR_ARG;
                    tot += v;
                }
                return tot > 0.0 ? MAPDEC_OK : MAPDEC_ERR_ARG;
            };
            st = read_prior(h.d.drift_start, h.phi0);
            if (!st) st = read_prior(h.d.drift_end, h.phiN);
            if (st) return st;
            h.d.drift_start = nullptr;
            h.d.drift_end = nullptr;
        }
        const bool per_sym = h.d.codebook_per_symbol != 0;
        if (h.d.codebook_per_symbol != 0 && h.d.codebook_per_symbol != 1) return MAPDEC_ERR_ARG;
        if (per_sym && (h.d.q > kPsMaxQ || (flags & MAPDEC_BATCH_SEGMENTED)))
            return MAPDEC_ERR_UNSUPPORTED;
        if (per_sym) {
            // N codebooks of q*n bytes, each injective (Sec. II-A)
            if (!h.d.codebook) return MAPDEC_ERR_ARG;
            const size_t cbn = (size_t)h.d.q * h.d.n;
            std::vector<uint8_t> all((size_t)h.d.N * cbn);
            if (is_device_ptr(h.d.codebook)) {
                CK(cudaMemcpy(all.data(), h.d.codebook, all.size(), cudaMemcpyDeviceToHost));
            } else {
                std::memcpy(all.data(), h.d.codebook, all.size());
            }
            h.cw.clear();
            h.cw.reserve((size_t)h.d.N * h.d.q);
            std::vector<uint32_t> one;
            for (int sym = 0; sym < h.d.N; ++sym) {
                st = pack_codebook(all.data() + (size_t)sym * cbn, h.d.q, h.d.n, one);
                if (st) return st;
                h.cw.insert(h.cw.end(), one.begin(), one.end());
            }
        } else {
            st = pack_codebook(h.d.codebook, h.d.q, h.d.n, h.cw);
            if (st) return st;
        }
        h.d.codebook = nullptr;
        const bool plain = (flags & MAPDEC_BATCH_PLAIN) != 0;
        mapdec_tune_t tu{};
        const bool tuned = !plain && tune_lookup(h.d.q, h.d.n, h.d.I, tu);
        plan_shape(h.dev, h.d, b->grad, plain ? 0 : forceP, tuned ? &tu : nullptr);
        h.store = tuned && tu.store_metric == 1;
        if (const char *e = std::getenv("MAPDEC_STORE_R")) h.store = std::atoi(e) == 1;  // testing
        if (plain || b->grad || (flags & MAPDEC_BATCH_SEGMENTED)) h.store = false;
        // tensor-core producers where the class supports it (default) in decode
        // mode.  Gradient batches keep the FP32 contractions: d logP / d(Pi, Pd,
        // Ps) is a sum of per-bit terms that nearly cancel, and the split-bf16 W
        // (about 2^-16 per product) leaves it 3e-4 off relative on small
        // gradients, where the FP32 W meets 1e-4.  MAPDEC_TC=0 keeps every frame
        // on the CUDA-core producers (A/B tests).
        // 0: the planner's rule, 1: wherever the class supports them, 2: never
        int tc_mode = tuned ? tu.tensor_cores : 0;
        if (const char *e = std::getenv("MAPDEC_TC")) tc_mode = std::atoi(e) != 0 ? 1 : 2;
        bool tc_on = tc_mode != 2;
        if (tuned && (tu.chain_threads == 128 || tu.chain_threads == 256 ||
                      tu.chain_threads == 512))
            b->chain_threads = tu.chain_threads;
        if (per_sym) {
            // per-symbol producers: work items (symbol, chunk of psC start states),
            // one APP partial row each (T2 * S2 rows with S2 = 1)
            FrameDev &f = h.dev;
            f.ps = 1;
            f.psC = ps_chunk_states(f.q, f.M);
            f.psT = (f.M + f.psC - 1) / f.psC;
            f.Tf = f.N * f.psT;
            f.T2 = f.N * f.psT;
            f.S2 = 1;
            h.store = false;
            tc_on = false;
        }
        h.tc = tc_on && !h.store && !b->grad && plan_fwd_tc(h.dev);
        if (h.tc && tc_mode == 0) {
            // the planner's rule: the tensor-core forward producer pays for its
            // per-tile work (bf16 splits, priors block, MMA wait) once a tile
            // spans many symbols, i.e. the CUDA-core contraction (S q per
            // (position, length)) outweighs the lattices (measured crossover)
            int smin = kTcMinSymbols;
            if (const char *e = std::getenv("MAPDEC_TC_MIN_S")) smin = std::atoi(e);
            if (h.dev.Sf < smin) {
                h.tc = false;
                h.dev.Pf = h.dev.P;
                h.dev.Sf = h.dev.S;
                h.dev.Tf = h.dev.T;
            }
        }
        if (h.tc) h.dev.Pgroups = prior_split_groups(h.dev);
        // the tensor-core APP producer only when asked for (it does not beat
        // the CUDA-core one on the mixed workload)
        bool tcb_on = tc_mode == 1;
        if (const char *e = std::getenv("MAPDEC_TC_BWD")) tcb_on = tc_on && std::atoi(e) != 0;
        h.tcb = tcb_on && h.tc && !b->grad && plan_bwd_tc(h.dev);
        if (flags & MAPDEC_BATCH_SEGMENTED) {
            int K = (int)std::ceil(std::sqrt((double)h.d.N));
            if (const char *e = std::getenv("MAPDEC_SEG_K")) {  // tuning / testing override
                const int k2 = std::atoi(e);
                if (k2 >= 1) K = k2;
            }
            K = std::max(1, std::min(K, h.d.N));
            h.segK = K;
            h.nseg = (h.d.N + K - 1) / K;
            h.scratch_floats = frame_scratch_floats_seg(h.dev, K, h.nseg, b->grad);
        } else {
            h.scratch_floats = frame_scratch_floats(h.dev, b->grad);
            if (h.store) h.scratch_floats += rup(metric_store_floats(h.dev), 64);
        }
        h.cost = frame_cost(h.dev);
        h.rx_off = b->rx_total;
        b->rx_total += h.d.rx_len;  // dense: the caller's concatenation, one copy
        h.sym_off = b->prior_total;  // element offset
        b->prior_total += (int64_t)h.d.N * h.d.q;
        h.rxw_off = b->rxw_total;
        b->rxw_total += (h.d.rx_len + 31) / 32 + 4;
        h.cw_off = b->cw_total;
        b->cw_total += (int64_t)h.cw.size();
        h.phi_off = b->phi_total;
        b->phi_total += (int64_t)(h.phi0.size() + h.phiN.size());
    }
    // resident buffers
    b->d_rx = (uint8_t *)b->dalloc(b->rx_total + 64);
    b->d_priors = (float *)b->dalloc(b->prior_total * 4);
    b->d_app = (float *)b->dalloc(b->prior_total * 4);
    if (b->grad) {
        b->d_dpriors = (float *)b->dalloc(b->prior_total * 4);
        b->d_dchan = (double *)b->dalloc((size_t)nf * 3 * 8);
    }
    if (flags & MAPDEC_BATCH_EXTRINSIC) b->d_ext = (float *)b->dalloc(b->prior_total * 4);
    b->d_loglik = (double *)b->dalloc((size_t)nf * 8);
    b->d_status = (int *)b->dalloc((size_t)nf * 4);
    b->d_rxw = (uint32_t *)b->dalloc(b->rxw_total * 4);
    b->d_cw = (uint32_t *)b->dalloc(b->cw_total * 4);
    {
        std::vector<uint32_t> cwall(b->cw_total);
        for (auto &h : b->fr) std::copy(h.cw.begin(), h.cw.end(), cwall.begin() + h.cw_off);
        CK(cudaMemcpy(b->d_cw, cwall.data(), cwall.size() * 4, cudaMemcpyHostToDevice));
    }
    if (b->phi_total > 0) {
        b->d_phi = (float *)b->dalloc((size_t)b->phi_total * 4);
        std::vector<float> all((size_t)b->phi_total);
        for (auto &h : b->fr) {
            std::copy(h.phi0.begin(), h.phi0.end(), all.begin() + h.phi_off);
            std::copy(h.phiN.begin(), h.phiN.end(), all.begin() + h.phi_off + h.phi0.size());
        }
        CK(cudaMemcpy(b->d_phi, all.data(), all.size() * 4, cudaMemcpyHostToDevice));
    }
    // Scratch budget and waves (frames kept in order; a wave is a contiguous
    // range).  If everything fits, one wave; otherwise waves rotate over three
    // scratch regions so that a wave's chains overlap the next wave's forward
    // producers and the previous wave's backward producers.
    size_t freeb = 0, totb = 0;
    CK(cudaMemGetInfo(&freeb, &totb));
    size_t bud = budget > 0 ? (size_t)budget : (size_t)(0.6 * (double)freeb);
    size_t maxf = 0, sumf = 0;
    for (auto &h : b->fr) { maxf = std::max(maxf, h.scratch_floats); sumf += h.scratch_floats; }
    const bool one_wave = sumf * 4 <= bud;
    size_t wave_bud = one_wave ? bud / 4 : bud / 4 / kRegions;  // in floats
    if (wave_bud < maxf) wave_bud = maxf;                        // at least one frame per wave
    {
        size_t acc = 0;
        Wave w;
        w.f0 = 0;
        for (int i = 0; i < nf; ++i) {
            if (acc + b->fr[i].scratch_floats > wave_bud && i > w.f0) {
                w.f1 = i;
                b->waves.push_back(w);
                w = Wave();
                w.f0 = i;
                acc = 0;
            }
            acc += b->fr[i].scratch_floats;
            b->scratch_floats = std::max(b->scratch_floats, acc);
        }
        w.f1 = nf;
        b->waves.push_back(w);
    }
    b->regions = b->waves.size() > 1 ? kRegions : 1;
    b->region_floats = rup(b->scratch_floats, 64);
    b->d_scratch = (float *)b->dalloc(b->region_floats * 4 * b->regions + 256);
    // per-wave descriptors and work tables
    const bool segmented = (flags & MAPDEC_BATCH_SEGMENTED) != 0;
    b->segmented = segmented;
    if (const char *e = std::getenv("MAPDEC_CHAIN_THREADS")) b->chain_threads = std::atoi(e);  // A/B override
    for (size_t wi = 0; wi < b->waves.size(); ++wi) {
        Wave &w = b->waves[wi];
        size_t off = (wi % b->regions) * b->region_floats;
        std::vector<FrameDev> devs;
        std::vector<const uint8_t *> rxp;
        std::vector<uint32_t *> rxwp;
        std::map<ClassKey, std::vector<int>> byclass;
        for (int i = w.f0; i < w.f1; ++i) {
            FrameHost &h = b->fr[i];
            FrameDev f = h.dev;
            f.rxbits = b->d_rxw + h.rxw_off;
            f.cw = b->d_cw + h.cw_off;
            f.phi0 = h.phi0.empty() ? nullptr : b->d_phi + h.phi_off;
            f.phiN = h.phiN.empty() ? nullptr : b->d_phi + h.phi_off + h.phi0.size();
            f.priors = b->d_priors + h.sym_off;
            float *base = b->d_scratch + off;
            size_t o = 0;
            f.Pbuf = nullptr;
            if (f.Pgroups) {
                f.Pbuf = reinterpret_cast<unsigned char *>(base + o);
                o += rup(prior_split_bytes(f) / 4, 64);
            }
            if (!segmented) {
                f.W = base + o; o += rup((size_t)f.N * f.wblk + 16, 64);
                f.alpha = base + o; o += rup((size_t)(f.N + 1) * f.Mp, 64);
                f.beta = base + o; o += rup((size_t)(f.N + 1) * f.Mp, 64);
                f.Lp = base + o; o += rup((size_t)f.T2 * f.S2 * f.q, 64);
                f.Gp = nullptr;
                if (b->grad) { f.Gp = base + o; o += rup((size_t)f.T2 * f.S2 * 3, 64); }
                f.thf = (double *)(base + o); o += rup((size_t)(f.N + 1) * 2, 64);
                f.mcf = (double *)(base + o); o += rup((size_t)(f.N + 1) * 2, 64);
                f.thb = (double *)(base + o); o += rup((size_t)(f.N + 1) * 2, 64);
                f.Gc = nullptr;
                if (b->grad) { f.Gc = (double *)(base + o); o += rup((size_t)finalize_chunks(f.N) * 3 * 2, 64); }
                f.Rg = nullptr;
                if (h.store) { f.Rg = base + o; o += rup(metric_store_floats(f), 64); }
            } else {
                // buffers of one segment; per-segment descriptors shift their bases
                const int K = h.segK, S = h.nseg;
                const int T2s = seg_supertiles(f, K), cps = finalize_chunks(K);
                // W, alpha and beta twice: segment s uses buffer s % 2, so a
                // segment's producers overlap the neighbouring segment's recursions
                f.W = base + o; o += 2 * rup((size_t)K * f.wblk + 16, 64);
                f.alpha = base + o; o += 2 * rup((size_t)(K + 1) * f.Mp, 64);
                f.beta = base + o; o += 2 * rup((size_t)(K + 1) * f.Mp, 64);
                f.Lp = base + o; o += rup((size_t)T2s * f.S2 * f.q, 64);
                f.Gp = nullptr;
                if (b->grad) { f.Gp = base + o; o += rup((size_t)T2s * f.S2 * 3, 64); }
                f.thf = (double *)(base + o); o += rup((size_t)(f.N + 1) * 2, 64);
                f.mcf = (double *)(base + o); o += rup((size_t)(f.N + 1) * 2, 64);
                f.thb = (double *)(base + o); o += rup((size_t)(f.N + 1) * 2, 64);
                f.Gc = nullptr;
                if (b->grad) { f.Gc = (double *)(base + o); o += rup((size_t)S * cps * 3 * 2, 64); }
                f.ckpt = base + o; o += rup((size_t)(S + 1) * f.Mp, 64);
                f.bedge = base + o; o += rup((size_t)f.Mp, 64);
                f.cst = (ChainState *)(base + o); o += rup(2 * chain_state_bytes() / 4 + 1, 64);
                f.chain_flags = CH_SEGMENTED;
                // chunk slots s*cps + c; only the last segment can be short
                f.fin_total = (S - 1) * cps + finalize_chunks(f.N - (S - 1) * K);
            }
            off += o;
            f.Rout = nullptr;
            f.app = b->d_app + h.sym_off;
            f.dpriors = b->grad ? b->d_dpriors + h.sym_off : nullptr;
            f.ext = b->d_ext ? b->d_ext + h.sym_off : nullptr;
            f.loglik = b->d_loglik + i;
            f.dchan = b->grad ? b->d_dchan + 3 * (size_t)i : nullptr;
            f.status = b->d_status + i;
            h.dev = f;
            devs.push_back(f);
            rxp.push_back(b->d_rx + h.rx_off);
            rxwp.push_back(b->d_rxw + h.rxw_off);
            w.max_words = std::max<long long>(w.max_words, (h.d.rx_len + 31) / 32 + 3);
            if (f.Pgroups)
                w.prior_split_threads = std::max<long long>(
                    w.prior_split_threads, (long long)f.Pgroups * (f.q / 8) * 8);
            byclass[ClassKey{h.d.n, h.d.I, (h.tc ? kTcFwd : 0) | (h.tcb ? kTcBwd : 0) |
                                               (f.ps ? kPerSym : 0)}]
                .push_back(i - w.f0);
        }
        const int nw = w.f1 - w.f0;
        w.d_frames = (FrameDev *)b->dalloc(sizeof(FrameDev) * nw);
        CK(cudaMemcpy(w.d_frames, devs.data(), sizeof(FrameDev) * nw, cudaMemcpyHostToDevice));
        w.d_rxptr = (const uint8_t **)b->dalloc(sizeof(void *) * nw);
        w.d_rxwptr = (uint32_t **)b->dalloc(sizeof(void *) * nw);
        CK(cudaMemcpy(w.d_rxptr, rxp.data(), sizeof(void *) * nw, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(w.d_rxwptr, rxwp.data(), sizeof(void *) * nw, cudaMemcpyHostToDevice));
        // chains: costliest frames first so long chains start early
        std::vector<int> order(nw);
        for (int k = 0; k < nw; ++k) order[k] = k;
        std::sort(order.begin(), order.end(), [&](int a, int c) {
            return (double)devs[a].N * devs[a].M * devs[a].MN >
                   (double)devs[c].N * devs[c].M * devs[c].MN;
        });
        std::vector<Work> chain;
        size_t csm = 0;
        for (int k : order) {
            chain.push_back({k, 0});
            chain.push_back({k, 1});
            csm = std::max(csm, chain_smem_bytes(devs[k]));
        }
        {
            std::vector<Work> fin;
            for (int k = 0; k < nw; ++k)
                for (int c = 0; c < finalize_chunks(devs[k].N); ++c) fin.push_back({k, c});
            w.nfin = (int)fin.size();
            w.d_fin = (Work *)b->dalloc(sizeof(Work) * fin.size());
            CK(cudaMemcpy(w.d_fin, fin.data(), sizeof(Work) * fin.size(), cudaMemcpyHostToDevice));
        }
        w.nchain = (int)chain.size();
        w.smem_chain = csm;
        w.d_chain = (Work *)b->dalloc(sizeof(Work) * chain.size());
        CK(cudaMemcpy(w.d_chain, chain.data(), sizeof(Work) * chain.size(), cudaMemcpyHostToDevice));
        for (auto &kv : byclass) {
            ClassLaunch c;
            c.n = std::get<0>(kv.first);
            c.I = std::get<1>(kv.first);
            c.tc = (std::get<2>(kv.first) & kTcFwd) != 0;
            c.tcb = (std::get<2>(kv.first) & kTcBwd) != 0;
            c.ps = (std::get<2>(kv.first) & kPerSym) != 0;
            std::vector<Work> fw, bw;
            for (int k : kv.second) {
                const FrameDev &f = devs[k];
                for (int t = 0; t < f.Tf; ++t) fw.push_back({k, t});
                for (int t = 0; t < f.T2; ++t) bw.push_back({k, t});
                c.smem_fwd = std::max(c.smem_fwd, c.tc ? fwd_tc_smem_bytes(f) : fwd_smem_bytes(f));
                c.smem_bwd = std::max(c.smem_bwd, c.ps    ? bwd_ps_smem_bytes(f, b->grad)
                                                  : c.tcb ? bwd_tc_smem_bytes(f)
                                                          : bwd_smem_bytes(f, b->grad));
            }
            c.nfwd = (int)fw.size();
            c.nbwd = (int)bw.size();
            c.d_fwd = (Work *)b->dalloc(sizeof(Work) * fw.size());
            c.d_bwd = (Work *)b->dalloc(sizeof(Work) * bw.size());
            CK(cudaMemcpy(c.d_fwd, fw.data(), sizeof(Work) * fw.size(), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c.d_bwd, bw.data(), sizeof(Work) * bw.size(), cudaMemcpyHostToDevice));
            w.cls.push_back(c);
        }
        if (segmented) build_segments(b, w, devs, byclass);
    }
    CK(cudaStreamCreateWithFlags(&b->aux_stream, cudaStreamNonBlocking));
    b->dep.resize(b->waves.size() * 2 + 2);
    for (auto &e : b->dep) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (flags & MAPDEC_BATCH_TIMING) {
        b->timing = true;
        b->events.resize(b->waves.size() * kPhases * 2);
        for (auto &e : b->events) CK(cudaEventCreate(&e));
    }
    return MAPDEC_OK;
}

// Enqueue one full run on stream st (producers) and the batch's auxiliary
// stream (chains).  The received bits of every wave are packed first.  Per
// wave w: forward producers on st; the chains
// on the auxiliary stream after the forward producers; the backward producers
// and finalize on st after the chains.  The forward producers of wave w+1 are
// issued before the backward producers of wave w, so they overlap wave w's
// chains; the three scratch regions keep overlapping waves apart.  With
// timing enabled, events bracket every phase of every wave (inside a captured
// graph they become external event nodes).  Throws CudaErr.
int64_t enqueue_run(mapdec_batch *b, bool grad, cudaStream_t st) {
    int64_t launches = 0;
    const int W = (int)b->waves.size();
    cudaStream_t cs = b->aux_stream;
    auto mark = [&](int w, int ph, int end, cudaStream_t s) {
        if (b->timing)
            CK(cudaEventRecordWithFlags(b->events[((size_t)w * kPhases + ph) * 2 + end], s,
                                        cudaEventRecordExternal));
    };
    cudaEvent_t fork = b->dep[2 * W], join = b->dep[2 * W + 1];
    CK(cudaMemsetAsync(b->d_status, 0, (size_t)b->nframes * 4, st));
    // received bits of every wave first (a batch-wide buffer): the packing
    // kernels then never wait behind recursions for a place on the GPU
    for (int w = 0; w < W; ++w) {
        Wave &wv = b->waves[w];
        mark(w, 0, 0, st);
        CK(launch_pack(wv.d_frames, wv.d_rxptr, wv.d_rxwptr, wv.f1 - wv.f0, wv.max_words, st));
        ++launches;
        mark(w, 0, 1, st);
    }
    CK(cudaEventRecord(fork, st));
    CK(cudaStreamWaitEvent(cs, fork, 0));
    auto forward = [&](int w) {
        Wave &wv = b->waves[w];
        mark(w, 1, 0, st);
        // the wave's priors split for the tensor-core producers, into the wave's
        // own scratch region (so only once its previous user is done with it)
        if (wv.prior_split_threads > 0) {
            CK(launch_prior_split(wv.d_frames, wv.f1 - wv.f0, wv.prior_split_threads, st));
            ++launches;
        }
        for (auto &c : wv.cls) {
            CK(c.ps   ? launch_fwd_ps(c.n, c.I, wv.d_frames, c.d_fwd, c.nfwd, st)
               : c.tc ? launch_fwd_tc(c.n, c.I, wv.d_frames, c.d_fwd, c.nfwd, c.smem_fwd, st)
                      : launch_fwd(c.n, c.I, wv.d_frames, c.d_fwd, c.nfwd, c.smem_fwd, st));
            ++launches;
        }
        mark(w, 1, 1, st);
        CK(cudaEventRecord(b->dep[2 * w], st));
        // chains of wave w on the auxiliary stream
        CK(cudaStreamWaitEvent(cs, b->dep[2 * w], 0));
        mark(w, 2, 0, cs);
        CK(launch_chain(wv.d_frames, wv.d_chain, wv.nchain, wv.smem_chain, b->chain_threads, cs));
        ++launches;
        mark(w, 2, 1, cs);
        CK(cudaEventRecord(b->dep[2 * w + 1], cs));
    };
    auto backward = [&](int w) {
        Wave &wv = b->waves[w];
        const int nw = wv.f1 - wv.f0;
        CK(cudaStreamWaitEvent(st, b->dep[2 * w + 1], 0));
        mark(w, 3, 0, st);
        for (auto &c : wv.cls) {
            CK(c.ps    ? launch_bwd_ps(c.n, c.I, grad, wv.d_frames, c.d_bwd, c.nbwd, c.smem_bwd, st)
               : c.tcb ? launch_bwd_tc(c.n, c.I, wv.d_frames, c.d_bwd, c.nbwd, c.smem_bwd, st)
                       : launch_bwd(c.n, c.I, grad, wv.d_frames, c.d_bwd, c.nbwd, c.smem_bwd, st));
            ++launches;
        }
        mark(w, 3, 1, st);
        mark(w, 4, 0, st);
        CK(launch_finalize(wv.d_frames, wv.d_fin, wv.nfin, nw, grad ? 1 : 0, st));
        launches += grad ? 2 : 1;
        mark(w, 4, 1, st);
    };
    forward(0);
    for (int w = 0; w < W; ++w) {
        if (w + 1 < W) forward(w + 1);
        backward(w);
    }
    CK(cudaEventRecord(join, cs));
    CK(cudaStreamWaitEvent(st, join, 0));
    return launches;
}

// Segmented run (checkpoint and recompute) on the producer stream st and the
// recursion stream.  Per wave: pack; a recording sweep over the segments in
// order (forward producers of the segment, then the forward recursions, which
// write the tilts and a checkpoint row at every segment boundary); then a sweep
// over the segments in reverse, each recomputing its W, replaying the forward
// recursion from its checkpoint with the recorded tilts (bit-identical rows)
// next to the backward recursion, then the APP producers and finalize of the
// segment.  W, alpha and beta are double-buffered by segment parity, so the
// producers of segment s+1 (s-1 in the second sweep) run while the
// recursions of segment s do; events keep every buffer's readers and writers
// in order.  The gradient chunks are added up after the last (first) segment.
// Timing phases: pack, recording-sweep producers (forward), all recursions
// (chains), recompute-sweep producers and finalize (backward); finalize reads 0.
int64_t enqueue_run_seg(mapdec_batch *b, bool grad, cudaStream_t st) {
    int64_t launches = 0;
    const int W = (int)b->waves.size();
    cudaStream_t cs = b->aux_stream;
    auto mark = [&](int w, int ph, int end, cudaStream_t s) {
        if (b->timing)
            CK(cudaEventRecordWithFlags(b->events[((size_t)w * kPhases + ph) * 2 + end], s,
                                        cudaEventRecordExternal));
    };
    cudaEvent_t fork = b->dep[2 * W], join = b->dep[2 * W + 1];
    CK(cudaMemsetAsync(b->d_status, 0, (size_t)b->nframes * 4, st));
    for (int w = 0; w < W; ++w) {
        Wave &wv = b->waves[w];
        const int nw = wv.f1 - wv.f0;
        const int S = (int)wv.segs.size();
        mark(w, 0, 0, st);
        CK(launch_pack(wv.d_frames, wv.d_rxptr, wv.d_rxwptr, nw, wv.max_words, st));
        ++launches;
        if (wv.prior_split_threads > 0) {
            CK(launch_prior_split(wv.d_frames, nw, wv.prior_split_threads, st));
            ++launches;
        }
        mark(w, 0, 1, st);
        CK(cudaEventRecord(fork, st));
        CK(cudaStreamWaitEvent(cs, fork, 0));
        mark(w, 1, 0, st);
        mark(w, 2, 0, cs);
        auto fwd = [&](SegLaunch &sl) {
            for (auto &c : sl.cls) {
                if (c.nfwd == 0) continue;
                CK(c.tc ? launch_fwd_tc(c.n, c.I, sl.d_frames, c.d_fwd, c.nfwd, c.smem_fwd, st)
                        : launch_fwd(c.n, c.I, sl.d_frames, c.d_fwd, c.nfwd, c.smem_fwd, st));
                ++launches;
            }
        };
        // recording sweep: fwd(s) on st once recording chain s-2 has read its buffer
        for (int s = 0; s < S; ++s) {
            SegLaunch &sl = wv.segs[s];
            if (s >= 2) CK(cudaStreamWaitEvent(st, wv.segs[s - 2].ev_rec, 0));
            fwd(sl);
            CK(cudaEventRecord(sl.ev_fwd, st));
            CK(cudaStreamWaitEvent(cs, sl.ev_fwd, 0));
            CK(launch_chain(sl.d_frames, sl.d_rec, sl.nrec, wv.smem_chain, b->chain_threads, cs));
            ++launches;
            CK(cudaEventRecord(sl.ev_rec, cs));
        }
        mark(w, 1, 1, st);
        // the recompute sweep reuses both buffers: every recording chain done
        CK(cudaStreamWaitEvent(st, wv.segs[S - 1].ev_rec, 0));
        mark(w, 3, 0, st);
        auto fwd2 = [&](int s) {
            SegLaunch &sl = wv.segs[s];
            // buffer s % 2 was last read by recompute-sweep chain s+2
            if (s + 2 < S) CK(cudaStreamWaitEvent(st, wv.segs[s + 2].ev_chain2, 0));
            fwd(sl);
            CK(cudaEventRecord(sl.ev_fwd2, st));
            CK(cudaStreamWaitEvent(cs, sl.ev_fwd2, 0));
            // alpha/beta buffer s % 2 was last read by the APP producers of segment s+2
            if (s + 2 < S) CK(cudaStreamWaitEvent(cs, wv.segs[s + 2].ev_bwd, 0));
            CK(launch_chain(sl.d_frames, sl.d_bw, sl.nbw, wv.smem_chain, b->chain_threads, cs));
            ++launches;
            CK(cudaEventRecord(sl.ev_chain2, cs));
        };
        fwd2(S - 1);
        for (int s = S - 1; s >= 0; --s) {
            SegLaunch &sl = wv.segs[s];
            if (s >= 1) fwd2(s - 1);  // overlaps the recursions of segment s
            CK(cudaStreamWaitEvent(st, sl.ev_chain2, 0));
            for (auto &c : sl.cls) {
                if (c.nbwd == 0) continue;
                CK(c.tcb ? launch_bwd_tc(c.n, c.I, sl.d_frames, c.d_bwd, c.nbwd, c.smem_bwd, st)
                         : launch_bwd(c.n, c.I, grad, sl.d_frames, c.d_bwd, c.nbwd, c.smem_bwd, st));
                ++launches;
            }
            CK(launch_finalize(sl.d_frames, sl.d_fin, sl.nfin, nw, grad ? 1 : 0, st,
                               grad && s == 0));
            launches += (grad && s == 0) ? 2 : 1;
            CK(cudaEventRecord(sl.ev_bwd, st));
        }
        mark(w, 2, 1, cs);
        CK(cudaEventRecord(join, cs));
        CK(cudaStreamWaitEvent(st, join, 0));
        mark(w, 3, 1, st);
        mark(w, 4, 0, st);
        mark(w, 4, 1, st);
    }
    return launches;
}

int64_t enqueue_any(mapdec_batch *b, bool grad, cudaStream_t st) {
    return b->segmented ? enqueue_run_seg(b, grad, st) : enqueue_run(b, grad, st);
}

int run_batch(mapdec_batch *b, bool grad) {
    if (grad && !b->grad) return MAPDEC_ERR_ARG;
    const bool use_graph = (b->flags & MAPDEC_BATCH_GRAPH) && !(b->flags & MAPDEC_BATCH_PLAIN);
    if (!use_graph) {
        b->last_launches = enqueue_any(b, grad, b->stream);
        return MAPDEC_OK;
    }
    if (!b->gexec || b->graph_grad != grad) {
        if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
        // the legacy default stream cannot be captured: capture on a private stream
        if (!b->cap_stream) CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        int64_t l = 0;
        try {
            l = enqueue_any(b, grad, b->cap_stream);
        } catch (CudaErr &e) {
            cudaStreamEndCapture(b->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        CK(cudaStreamEndCapture(b->cap_stream, &g));
        cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        b->graph_grad = grad;
        b->launches_per_run[grad ? 1 : 0] = l;
    }
    CK(cudaGraphLaunch(b->gexec, b->stream));
    b->last_launches = b->launches_per_run[grad ? 1 : 0];
    return MAPDEC_OK;
}

int worst_status(mapdec_batch *b) {
    std::vector<int> st(b->nframes);
    CK(cudaMemcpyAsync(st.data(), b->d_status, st.size() * 4, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    int w = 0;
    for (int s : st) w = std::max(w, s);
    return w;
}

// Copy inputs (host or device) into the resident buffers.
void load_inputs(mapdec_batch *b, const uint8_t *rx_all, const float *priors_all) {
    cudaStream_t st = b->stream;
    if (rx_all) copy_in(b->d_rx, rx_all, (size_t)b->rx_total, st);
    if (priors_all) {
        copy_in(b->d_priors, priors_all, (size_t)b->prior_total * 4, st);
    } else {
        // uniform priors: 1/q per frame
        std::vector<float> u((size_t)b->prior_total);
        for (auto &h : b->fr)
            std::fill(u.begin() + h.sym_off, u.begin() + h.sym_off + (size_t)h.d.N * h.d.q,
                      1.0f / (float)h.d.q);
        CK(cudaMemcpyAsync(b->d_priors, u.data(), u.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
}

}  // namespace


// ---------------------------------------------------------------------------
// Allocation-free decode of one frame.
//
// Some callers cannot allocate device memory once they are running: a
// receiver pipeline whose memory is fixed at start-up, a host framework that
// owns every device allocation itself, or real-time code that must not risk a
// cudaMalloc blocking, fragmenting or failing in mid-stream.  For them the
// whole scratch of one decode (descriptor, work lists, packed bits, W, alpha,
// beta, APP partial sums, status) is carved out of the file-scope array
// below, which every GPU that loads the library holds until the process
// exits.  Nothing is allocated per call, on the device or on the host.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kStaticMaxQ = 64;
constexpr int kStaticMaxDevices = 64;

struct StaticCodebook {
    uint32_t w[kStaticMaxQ];
};

std::mutex g_static_mu;
void *g_static_addr[kStaticMaxDevices] = {};

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

// Device address of the static arena on the current device.  The host-side
// name g_static_scratch is only a stand-in; the address is looked up once per
// device with that device current.
int static_scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MAPDEC_ERR_CUDA;
    }
    if (dev < 0 || dev >= kStaticMaxDevices) return MAPDEC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return MAPDEC_ERR_CUDA;
        }
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return MAPDEC_OK;
}

// Writes the descriptor, work lists and pointer tables into the arena, fills
// uniform priors if none were given, and clears the status word (the arena
// keeps the previous call's contents).
__global__ void k_static_setup(FrameDev f, FrameDev *fdst, Work *fwd, int T, Work *bwd, int T2,
                               Work *chain, Work *fin, int nfin, const uint8_t **rxp,
                               uint32_t **rxwp,
                               const uint8_t *rx, uint32_t *rxw, uint32_t *cwdst,
                               StaticCodebook cb, int q, float *uni, long long nuni,
                               float uval, int *status) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long t = tid; t < T; t += nth) fwd[t] = Work{0, (int)t};
    for (long long t = tid; t < T2; t += nth) bwd[t] = Work{0, (int)t};
    for (long long c = tid; c < nfin; c += nth) fin[c] = Work{0, (int)c};
    for (long long k = tid; k < nuni; k += nth) uni[k] = uval;
    for (long long d = tid; d < q; d += nth) cwdst[d] = cb.w[d];
    if (tid == 0) {
        *fdst = f;
        chain[0] = Work{0, 0};
        chain[1] = Work{0, 1};
        rxp[0] = rx;
        rxwp[0] = rxw;
        *status = 0;
    }
}

bool device_pointer(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *mapdec_strerror(int s) {
    switch (s) {
        case MAPDEC_OK: return "ok";
        case MAPDEC_ERR_ARG: return "invalid argument";
        case MAPDEC_ERR_DRIFT_RANGE: return "received length outside the drift limit";
        case MAPDEC_ERR_ZERO_PROB: return "no channel path within the drift limits explains the received bits";
        case MAPDEC_ERR_NOMEM: return "out of memory";
        case MAPDEC_ERR_CUDA: return "CUDA error or no usable device";
        case MAPDEC_ERR_TIMEOUT: return "device-side wait timed out";
        case MAPDEC_ERR_UNSUPPORTED: return "parameters outside the supported range";
        case MAPDEC_ERR_TOO_LARGE: return "frame needs more scratch than the static arena of mapdec_decode_noalloc holds";
        default: return "unknown status";
    }
}

int mapdec_batch_create(mapdec_batch_t **out, const mapdec_frame_desc_t *frames, int num_frames,
                        int flags, int64_t mem_budget_bytes) {
    if (!out || !frames || num_frames < 1) return MAPDEC_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return MAPDEC_ERR_CUDA;
    }
    mapdec_batch *b = new (std::nothrow) mapdec_batch();
    if (!b) return MAPDEC_ERR_NOMEM;
    int forceP = 0;
    if (const char *e = std::getenv("MAPDEC_FORCE_P")) forceP = std::atoi(e);
    int st;
    try {
        st = build_batch(b, frames, num_frames, flags, mem_budget_bytes, forceP);
    } catch (CudaErr &e) {
        cudaGetLastError();
        st = map_cuda(e.e);
    } catch (std::bad_alloc &) {
        st = MAPDEC_ERR_NOMEM;
    }
    if (st != MAPDEC_OK) {
        delete b;
        return st;
    }
    *out = b;
    return MAPDEC_OK;
}

int mapdec_batch_layout(mapdec_batch_t *b, int64_t *rx_offsets, int64_t *sym_offsets,
                        int64_t *rx_total, int64_t *prior_elems_total) {
    if (!b) return MAPDEC_ERR_ARG;
    int64_t acc = 0;
    for (int i = 0; i < b->nframes; ++i) {
        if (rx_offsets) rx_offsets[i] = acc;
        acc += b->fr[i].d.rx_len;
        if (sym_offsets) sym_offsets[i] = b->fr[i].sym_off;
    }
    if (rx_total) *rx_total = acc;
    if (prior_elems_total) *prior_elems_total = b->prior_total;
    return MAPDEC_OK;
}

int mapdec_batch_buffers(mapdec_batch_t *b, uint8_t **rx_dev, float **priors_dev, float **app_dev,
                         double **loglik_dev) {
    if (!b) return MAPDEC_ERR_ARG;
    if (rx_dev) *rx_dev = b->d_rx;
    if (priors_dev) *priors_dev = b->d_priors;
    if (app_dev) *app_dev = b->d_app;
    if (loglik_dev) *loglik_dev = b->d_loglik;
    return MAPDEC_OK;
}

int64_t mapdec_batch_rx_offset(mapdec_batch_t *b, int frame) {
    if (!b || frame < 0 || frame >= b->nframes) return -1;
    return b->fr[frame].rx_off;
}

int mapdec_batch_run(mapdec_batch_t *b) {
    if (!b) return MAPDEC_ERR_ARG;
    try {
        return run_batch(b, false);
    } catch (CudaErr &e) {
        cudaGetLastError();
        return map_cuda(e.e);
    }
}

int mapdec_batch_sync(mapdec_batch_t *b) {
    if (!b) return MAPDEC_ERR_ARG;
    try {
        return worst_status(b);
    } catch (CudaErr &e) {
        cudaGetLastError();
        return map_cuda(e.e);
    }
}

int mapdec_batch_status(mapdec_batch_t *b, int *status_per_frame) {
    if (!b || !status_per_frame) return MAPDEC_ERR_ARG;
    if (cudaMemcpy(status_per_frame, b->d_status, (size_t)b->nframes * 4,
                   cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return MAPDEC_ERR_CUDA;
    }
    return MAPDEC_OK;
}

int mapdec_batch_decode(mapdec_batch_t *b, const uint8_t *rx_all, const float *priors_all,
                        float *app_all, double *loglik_all) {
    if (!b || !rx_all) return MAPDEC_ERR_ARG;
    try {
        load_inputs(b, rx_all, priors_all);
        int st = run_batch(b, false);
        if (st) return st;
        copy_out(app_all, b->d_app, (size_t)b->prior_total * 4, b->stream);
        copy_out(loglik_all, b->d_loglik, (size_t)b->nframes * 8, b->stream);
        return worst_status(b);
    } catch (CudaErr &e) {
        cudaGetLastError();
        return map_cuda(e.e);
    }
}

int mapdec_batch_decode_ext(mapdec_batch_t *b, const uint8_t *rx_all, const float *priors_all,
                            float *app_all, float *ext_all, double *loglik_all) {
    if (!b || !rx_all || !b->d_ext) return MAPDEC_ERR_ARG;
    try {
        load_inputs(b, rx_all, priors_all);
        int st = run_batch(b, false);
        if (st) return st;
        copy_out(app_all, b->d_app, (size_t)b->prior_total * 4, b->stream);
        copy_out(ext_all, b->d_ext, (size_t)b->prior_total * 4, b->stream);
        copy_out(loglik_all, b->d_loglik, (size_t)b->nframes * 8, b->stream);
        return worst_status(b);
    } catch (CudaErr &e) {
        cudaGetLastError();
        return map_cuda(e.e);
    }
}

int mapdec_batch_loglik_grad(mapdec_batch_t *b, const uint8_t *rx_all, const float *priors_all,
                             double *dchan_all, float *dpriors_all, double *loglik_all) {
    if (!b || !rx_all) return MAPDEC_ERR_ARG;
    if (!b->grad) return MAPDEC_ERR_ARG;
    try {
        load_inputs(b, rx_all, priors_all);
        int st = run_batch(b, true);
        if (st) return st;
        copy_out(dchan_all, b->d_dchan, (size_t)b->nframes * 3 * 8, b->stream);
        copy_out(dpriors_all, b->d_dpriors, (size_t)b->prior_total * 4, b->stream);
        copy_out(loglik_all, b->d_loglik, (size_t)b->nframes * 8, b->stream);
        return worst_status(b);
    } catch (CudaErr &e) {
        cudaGetLastError();
        return map_cuda(e.e);
    }
}

int mapdec_batch_set_stream(mapdec_batch_t *b, void *s) {
    if (!b) return MAPDEC_ERR_ARG;
    b->stream = (cudaStream_t)s;
    return MAPDEC_OK;
}

void mapdec_batch_destroy(mapdec_batch_t *b) { delete b; }

int64_t mapdec_batch_last_launches(mapdec_batch_t *b) { return b ? b->last_launches : -1; }

int mapdec_batch_phase_ms(mapdec_batch_t *b, double *ms) {
    if (!b || !ms) return MAPDEC_ERR_ARG;
    if (!b->timing) return MAPDEC_ERR_ARG;
    for (int k = 0; k < kPhases; ++k) ms[k] = 0.0;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return MAPDEC_ERR_CUDA;
    }
    for (size_t w = 0; w < b->waves.size(); ++w)
        for (int k = 0; k < kPhases; ++k) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, b->events[(w * kPhases + k) * 2],
                                     b->events[(w * kPhases + k) * 2 + 1]) != cudaSuccess) {
                cudaGetLastError();
                return MAPDEC_ERR_CUDA;
            }
            ms[k] += t;
        }
    return MAPDEC_OK;
}

int mapdec_batch_num_waves(mapdec_batch_t *b) { return b ? (int)b->waves.size() : -1; }

int mapdec_batch_tc_frames(mapdec_batch_t *b, int *flags) {
    if (!b) return -1;
    int c = 0;
    for (size_t k = 0; k < b->fr.size(); ++k) {
        const FrameHost &h = b->fr[k];
        c += h.tc ? 1 : 0;
        if (flags) flags[k] = (h.tc ? 1 : 0) | (h.tcb ? 2 : 0);
    }
    return c;
}

int mapdec_tune_set(int q, int n, int I, const mapdec_tune_t *t) {
    if (q < 2 || n < 1 || I < 1) return MAPDEC_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (size_t k = 0; k < g_tune.size(); ++k)
        if (g_tune[k].q == q && g_tune[k].n == n && g_tune[k].I == I) {
            if (t) g_tune[k].t = *t;
            else g_tune.erase(g_tune.begin() + (long)k);
            return MAPDEC_OK;
        }
    if (t) g_tune.push_back({q, n, I, *t});
    return MAPDEC_OK;
}

int mapdec_tune_get(int q, int n, int I, mapdec_tune_t *t) {
    if (!t) return MAPDEC_ERR_ARG;
    return tune_lookup(q, n, I, *t) ? MAPDEC_OK : MAPDEC_ERR_ARG;
}

int mapdec_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    return MAPDEC_OK;
}

// ---------------------------------------------------------------------------
// single-frame handle
// ---------------------------------------------------------------------------
int mapdec_create(mapdec_t **out, int q, int n, const uint8_t *codebook, int N, double Pi,
                  double Pd, double Ps, int I, int xmax) {
    if (!out) return MAPDEC_ERR_ARG;
    *out = nullptr;
    int st = validate(q, n, N, Pi, Pd, Ps, I, xmax);
    if (st) return st;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return MAPDEC_ERR_CUDA;
    }
    std::vector<uint32_t> cw;
    st = pack_codebook(codebook, q, n, cw);
    if (st) return st;
    mapdec *h = new (std::nothrow) mapdec();
    if (!h) return MAPDEC_ERR_NOMEM;
    h->q = q; h->n = n; h->N = N; h->I = I; h->xmax = xmax;
    h->Pi = Pi; h->Pd = Pd; h->Ps = Ps;
    h->rho_max = (int64_t)n * N + xmax;
    h->codebook.resize((size_t)q * n);
    for (int d = 0; d < q; ++d)
        for (int r = 0; r < n; ++r) h->codebook[(size_t)d * n + r] = (cw[d] >> r) & 1u;
    mapdec_frame_desc_t d;
    d.q = q; d.n = n; d.N = N; d.I = I; d.xmax = xmax;
    d.Pi = Pi; d.Pd = Pd; d.Ps = Ps;
    d.codebook = h->codebook.data();
    d.rx_len = h->rho_max;
    d.codebook_per_symbol = 0;
    d.drift_start = nullptr;
    d.drift_end = nullptr;
    st = mapdec_batch_create(&h->b, &d, 1, MAPDEC_BATCH_PLAIN | MAPDEC_BATCH_EXTRINSIC, 0);
    if (st) {
        delete h;
        return st;
    }
    if (cudaMalloc(&h->d_phi, (size_t)2 * (2 * xmax + 1) * 4) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return MAPDEC_ERR_NOMEM;
    }
    *out = h;
    return MAPDEC_OK;
}

int mapdec_set_stream(mapdec_t *h, void *s) {
    if (!h) return MAPDEC_ERR_ARG;
    h->stream = (cudaStream_t)s;
    if (h->b) h->b->stream = h->stream;
    if (h->bg) h->bg->stream = h->stream;
    return MAPDEC_OK;
}

namespace {

// Point the one-frame batch of a handle at received length rho (allocated for
// rho_max >= rho): the descriptor gets rho and its tile counts, the producer
// launches their prefix of the work lists, and the extrinsic output pointer is
// set only when asked for.  Nothing is allocated.
void retarget_single(mapdec_batch *b, int64_t rho, bool ext, const float *phi0,
                     const float *phiN) {
    FrameHost &h = b->fr[0];
    FrameDev &f = h.dev;
    f.phi0 = phi0;
    f.phiN = phiN;
    h.d.rx_len = rho;
    f.rho = rho;
    if (!f.ps) {  // per-symbol work items do not depend on rho
        f.T = (int)((rho + 1 + f.P - 1) / f.P);
        f.T2 = (f.T + f.nsub - 1) / f.nsub;
        f.Tf = (int)((rho + 1 + f.Pf - 1) / f.Pf);
    }
    f.ext = ext ? b->d_ext : nullptr;
    b->rx_total = rho;
    Wave &w = b->waves[0];
    for (auto &c : w.cls) {
        c.nfwd = f.Tf;
        c.nbwd = f.T2;
    }
    CK(cudaMemcpyAsync(w.d_frames, &f, sizeof(FrameDev), cudaMemcpyHostToDevice, b->stream));
}

}  // namespace

static int ensure_single(mapdec_t *h, int64_t rho, bool grad, bool ext = false) {
    const long long tau = (long long)h->n * h->N;
    if (rho < 0) return MAPDEC_ERR_ARG;
    if (std::llabs(rho - tau) > h->xmax) return MAPDEC_ERR_DRIFT_RANGE;
    if (grad && !h->bg) {
        mapdec_frame_desc_t d;
        d.q = h->q; d.n = h->n; d.N = h->N; d.I = h->I; d.xmax = h->xmax;
        d.Pi = h->Pi; d.Pd = h->Pd; d.Ps = h->Ps;
        d.codebook = h->codebook.data();
        d.rx_len = h->rho_max;
        d.codebook_per_symbol = 0;
        d.drift_start = nullptr;
        d.drift_end = nullptr;
        int st = mapdec_batch_create(&h->bg, &d, 1, MAPDEC_BATCH_PLAIN | MAPDEC_BATCH_GRAD, 0);
        if (st) return st;
        h->bg->stream = h->stream;
    }
    try {
        const int M = 2 * h->xmax + 1;
        retarget_single(grad ? h->bg : h->b, rho, ext, h->use_phi0 ? h->d_phi : nullptr,
                        h->use_phiN ? h->d_phi + M : nullptr);
    } catch (CudaErr &e) {
        cudaGetLastError();
        return map_cuda(e.e);
    }
    return MAPDEC_OK;
}

int mapdec_decode(mapdec_t *h, const uint8_t *rx, int64_t rx_len, const float *priors,
                  float *app_out, double *loglik_out) {
    if (!h || (!rx && rx_len > 0)) return MAPDEC_ERR_ARG;
    int st = ensure_single(h, rx_len, false);
    if (st) return st;
    return mapdec_batch_decode(h->b, rx ? rx : (const uint8_t *)"", priors, app_out, loglik_out);
}

int mapdec_decode_ext(mapdec_t *h, const uint8_t *rx, int64_t rx_len, const float *priors,
                      float *app_out, float *ext_out, double *loglik_out) {
    if (!h || (!rx && rx_len > 0)) return MAPDEC_ERR_ARG;
    int st = ensure_single(h, rx_len, false, true);
    if (st) return st;
    return mapdec_batch_decode_ext(h->b, rx ? rx : (const uint8_t *)"", priors, app_out, ext_out,
                                   loglik_out);
}

int mapdec_loglik_grad(mapdec_t *h, const uint8_t *rx, int64_t rx_len, const float *priors,
                       double *dlogp_dchan, float *dlogp_dpriors, double *loglik_out) {
    if (!h || (!rx && rx_len > 0)) return MAPDEC_ERR_ARG;
    if (!(h->Pd > 0) || !((1.0 - h->Pi - h->Pd) * (1.0 - h->Ps) > 0)) return MAPDEC_ERR_UNSUPPORTED;
    int st = ensure_single(h, rx_len, true);
    if (st) return st;
    return mapdec_batch_loglik_grad(h->bg, rx ? rx : (const uint8_t *)"", priors, dlogp_dchan,
                                    dlogp_dpriors, loglik_out);
}

int mapdec_receiver_metric(mapdec_t *h, const uint8_t *rx, int64_t rx_len, float *R_out) {
    if (!h || !R_out || (!rx && rx_len > 0)) return MAPDEC_ERR_ARG;
    int st = ensure_single(h, rx_len, false);
    if (st) return st;
    mapdec_batch *b = h->b;
    try {
        load_inputs(b, rx ? rx : (const uint8_t *)"", nullptr);
        const FrameHost &fh = b->fr[0];
        if (!h->d_rout)
            CK(cudaMalloc(&h->d_rout, (size_t)(h->rho_max + 1) * h->q * fh.dev.MN * 4));
        const size_t nfl = (size_t)(rx_len + 1) * h->q * fh.dev.MN;
        Wave &w = b->waves[0];
        FrameDev f = fh.dev;
        f.Rout = h->d_rout;
        CK(cudaMemcpyAsync(w.d_frames, &f, sizeof(FrameDev), cudaMemcpyHostToDevice, b->stream));
        CK(launch_pack(w.d_frames, w.d_rxptr, w.d_rxwptr, 1, w.max_words, b->stream));
        CK(launch_rmetric(h->n, h->I, w.d_frames, (long long)(rx_len + 1) * h->q, b->stream));
        CK(cudaMemcpyAsync(w.d_frames, &fh.dev, sizeof(FrameDev), cudaMemcpyHostToDevice, b->stream));
        copy_out(R_out, h->d_rout, nfl * 4, b->stream);
        CK(cudaStreamSynchronize(b->stream));
        return MAPDEC_OK;
    } catch (CudaErr &e) {
        cudaGetLastError();
        return map_cuda(e.e);
    }
}

int mapdec_set_drift_priors(mapdec_t *h, const float *drift_start, const float *drift_end) {
    if (!h) return MAPDEC_ERR_ARG;
    const int M = 2 * h->xmax + 1;
    std::vector<float> v((size_t)M);
    const float *src[2] = {drift_start, drift_end};
    for (int k = 0; k < 2; ++k) {
        if (!src[k]) continue;
        if (is_device_ptr(src[k])) {
            if (cudaMemcpy(v.data(), src[k], (size_t)M * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
                cudaGetLastError();
                return MAPDEC_ERR_CUDA;
            }
        } else {
            std::memcpy(v.data(), src[k], (size_t)M * 4);
        }
        double tot = 0.0;
        for (float x : v) {
            if (!(x >= 0.f) || !std::isfinite(x)) return MAPDEC_ERR_ARG;
            tot += x;
        }
        if (!(tot > 0.0)) return MAPDEC_ERR_ARG;
        if (cudaMemcpy(h->d_phi + (size_t)k * M, v.data(), (size_t)M * 4,
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return MAPDEC_ERR_CUDA;
        }
    }
    h->use_phi0 = drift_start != nullptr;
    h->use_phiN = drift_end != nullptr;
    return MAPDEC_OK;
}

void mapdec_destroy(mapdec_t *h) { delete h; }

int mapdec_decode_noalloc(const mapdec_frame_desc_t *frame, const uint8_t *rx_dev,
                          const float *priors_dev, float *app_dev, double *loglik_dev,
                          void *cuda_stream) {
    if (!frame || !app_dev || !loglik_dev) return MAPDEC_ERR_ARG;
    const mapdec_frame_desc_t &d = *frame;
    int st = validate(d.q, d.n, d.N, d.Pi, d.Pd, d.Ps, d.I, d.xmax);
    if (st) return st;
    if (d.codebook_per_symbol || d.drift_start || d.drift_end) return MAPDEC_ERR_UNSUPPORTED;
    if (d.q > kStaticMaxQ) return MAPDEC_ERR_TOO_LARGE;
    const long long tau = (long long)d.n * d.N;
    if (d.rx_len < 0) return MAPDEC_ERR_ARG;
    if (std::llabs(d.rx_len - tau) > d.xmax) return MAPDEC_ERR_DRIFT_RANGE;
    if ((d.rx_len > 0 && !device_pointer(rx_dev)) || !device_pointer(app_dev) ||
        !device_pointer(loglik_dev) || (priors_dev && !device_pointer(priors_dev)))
        return MAPDEC_ERR_ARG;
    // codebook: host or device bytes, copied into a stack buffer and packed
    if (!d.codebook) return MAPDEC_ERR_ARG;
    uint8_t cbytes[kStaticMaxQ * 31];
    const size_t cbn = (size_t)d.q * d.n;
    if (device_pointer(d.codebook)) {
        if (cudaMemcpy(cbytes, d.codebook, cbn, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return MAPDEC_ERR_CUDA;
        }
    } else {
        std::memcpy(cbytes, d.codebook, cbn);
    }
    StaticCodebook cb;
    for (int k = 0; k < d.q; ++k) {
        uint32_t w = 0;
        for (int r = 0; r < d.n; ++r) {
            const uint8_t bit = cbytes[(size_t)k * d.n + r];
            if (bit > 1) return MAPDEC_ERR_ARG;
            if (bit) w |= (1u << r);
        }
        for (int k2 = 0; k2 < k; ++k2)
            if (cb.w[k2] == w) return MAPDEC_ERR_ARG;  // the encoding must be injective
        cb.w[k] = w;
    }
    void *base = nullptr;
    st = static_scratch_address(&base);
    if (st) return st;

    FrameDev f{};
    plan_shape(f, d, false, 0);
    // carve the arena (every region 256-byte aligned)
    size_t off = 0;
    auto take = [&](size_t bytes) -> size_t {
        const size_t o = off;
        off += rup(bytes, 256);
        return o;
    };
    const size_t o_frame = take(sizeof(FrameDev));
    const size_t o_fwd = take(sizeof(Work) * (size_t)f.Tf);
    const size_t o_bwd = take(sizeof(Work) * (size_t)f.T2);
    const size_t o_chain = take(sizeof(Work) * 2);
    const int nfin = finalize_chunks(d.N);
    const size_t o_fin = take(sizeof(Work) * (size_t)nfin);
    const size_t o_rxp = take(sizeof(void *));
    const size_t o_rxwp = take(sizeof(void *));
    const long long nwords = (d.rx_len + 31) / 32 + 4;
    const size_t o_rxw = take(4 * (size_t)nwords);
    const size_t o_cw = take(4 * (size_t)d.q);
    const size_t o_pri = priors_dev ? off : take(4 * (size_t)d.N * d.q);
    const size_t o_W = take(4 * ((size_t)f.N * f.wblk + 16));
    const size_t o_a = take(4 * (size_t)(f.N + 1) * f.Mp);
    const size_t o_b = take(4 * (size_t)(f.N + 1) * f.Mp);
    const size_t o_Lp = take(4 * (size_t)f.T2 * f.S2 * f.q);
    const size_t o_thf = take(8 * (size_t)(f.N + 1));
    const size_t o_mcf = take(8 * (size_t)(f.N + 1));
    const size_t o_thb = take(8 * (size_t)(f.N + 1));
    const size_t o_st = take(sizeof(int));
    if (off > kStaticScratchBytes) return MAPDEC_ERR_TOO_LARGE;

    unsigned char *A = (unsigned char *)base;
    f.rxbits = (const uint32_t *)(A + o_rxw);
    f.cw = (const uint32_t *)(A + o_cw);
    f.priors = priors_dev ? priors_dev : (const float *)(A + o_pri);
    f.W = (float *)(A + o_W);
    f.alpha = (float *)(A + o_a);
    f.beta = (float *)(A + o_b);
    f.Lp = (float *)(A + o_Lp);
    f.thf = (double *)(A + o_thf);
    f.mcf = (double *)(A + o_mcf);
    f.thb = (double *)(A + o_thb);
    f.Gp = nullptr;
    f.Gc = nullptr;
    f.Rout = nullptr;
    f.app = app_dev;
    f.dpriors = nullptr;
    f.loglik = loglik_dev;
    f.dchan = nullptr;
    f.status = (int *)(A + o_st);

    cudaStream_t s = (cudaStream_t)cuda_stream;
    FrameDev *fdev = (FrameDev *)(A + o_frame);
    Work *wf = (Work *)(A + o_fwd), *wb = (Work *)(A + o_bwd), *wc = (Work *)(A + o_chain);
    Work *wfin = (Work *)(A + o_fin);
    const long long nuni = priors_dev ? 0 : (long long)d.N * d.q;
    k_static_setup<<<64, 256, 0, s>>>(f, fdev, wf, f.Tf, wb, f.T2, wc, wfin, nfin,
                                      (const uint8_t **)(A + o_rxp), (uint32_t **)(A + o_rxwp),
                                      rx_dev, (uint32_t *)(A + o_rxw), (uint32_t *)(A + o_cw), cb,
                                      d.q, (float *)(A + o_pri), nuni, 1.0f / (float)d.q,
                                      f.status);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_pack(fdev, (const uint8_t *const *)(A + o_rxp), (uint32_t *const *)(A + o_rxwp), 1,
                        nwords, s);
    if (e == cudaSuccess) e = launch_fwd(d.n, d.I, fdev, wf, f.Tf, fwd_smem_bytes(f), s);
    if (e == cudaSuccess) e = launch_chain(fdev, wc, 2, chain_smem_bytes(f), 0, s);
    if (e == cudaSuccess) e = launch_bwd(d.n, d.I, false, fdev, wb, f.T2, bwd_smem_bytes(f, false), s);
    if (e == cudaSuccess) e = launch_finalize(fdev, wfin, nfin, 1, 0, s);
    int status = MAPDEC_OK;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, f.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return map_cuda(e);
    }
    return status;
}

}  // extern "C"
