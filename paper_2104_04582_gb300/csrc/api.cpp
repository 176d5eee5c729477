// api.cpp -- host side of libfewsum.so: the C ABI declared in include/fewsum.h.
//
// Responsibilities: input validation, the planning step (mode -> harmonic slot layout,
// segment sample ranges, CTA slices of equal pass cost), device memory from a context-owned
// stream-ordered pool with an HBM budget, plan uploads through pinned staging buffers, kernel
// launches, CUDA-graph capture of batches, and the device error latch.  No arithmetic of the
// waveform itself happens here; every numerical step runs in the kernels.
#include "../../include/fewsum.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "fewsum_internal.h"

using namespace fewsum;

// ------------------------------------------------------------------------------ utilities

namespace {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

#define FEW_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) {                           \
            (void)cudaGetLastError();                       \
            return e__ == cudaErrorMemoryAllocation ? FEW_ERR_NOMEM : FEW_ERR_CUDA; \
        }                                                   \
    } while (0)

// Pinned host staging blocks for plan uploads, reused once their copy has completed.
struct PinnedPool {
    struct Block {
        void *p = nullptr;
        size_t bytes = 0;
        cudaEvent_t ev = nullptr;
        bool pending = false;
    };
    std::vector<Block> blocks;

    ~PinnedPool() { release(); }
    void release()
    {
        for (auto &b : blocks) {
            if (b.ev) cudaEventDestroy(b.ev);
            if (b.p) cudaFreeHost(b.p);
        }
        blocks.clear();
    }
    // A block of at least `bytes` that no queued copy still reads.
    Block *acquire(size_t bytes)
    {
        for (auto &b : blocks) {
            if (b.bytes < bytes) continue;
            if (b.pending) {
                if (cudaEventQuery(b.ev) != cudaSuccess) continue;
                b.pending = false;
            }
            return &b;
        }
        Block nb;
        nb.bytes = align_up(std::max(bytes, (size_t)1 << 16), 4096);
        if (cudaHostAlloc(&nb.p, nb.bytes, cudaHostAllocDefault) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        if (cudaEventCreateWithFlags(&nb.ev, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaFreeHost(nb.p);
            return nullptr;
        }
        blocks.push_back(nb);
        return &blocks.back();
    }
};

}  // namespace

struct few_traj;
struct few_batch;

struct few_ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;  // 0: unlimited
    size_t in_use = 0;
    cudaMemPool_t pool = nullptr;
    cudaStream_t internal = nullptr;
    // second streams for work beside a call's main chain (the phase anchors beside the
    // harmonics and the fold; the reduced-basis scale beside its pack), each with its fork and
    // join events; taken in turn, so calls on different user streams seldom share one
    struct SideLane {
        cudaStream_t s = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
    } lanes[4];
    unsigned lane_next = 0;
    unsigned *d_err = nullptr;
    std::recursive_mutex mu;
    std::unordered_map<void *, size_t> sizes;
    std::set<few_traj *> trajs;
    std::set<few_batch *> batches;
    std::set<few_basis *> bases;
    PinnedPool pinned;
    int tile_R[2] = {1, 8};
    int tile_T[2] = {256, 256};
    int tile_S[2] = {256, 1024};  // slots per ring stage (the mode tile)
    std::map<std::tuple<int, int, int, int>, int> occ_cache;
    bool timing = false;
    cudaEvent_t tev[8] = {};
    bool trec[4] = {false, false, false, false};
};

namespace {

// A named NVTX range over an entry point's host work (inert unless a profiler is attached), so a
// timeline shows which call queued which kernels.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

few_status dev_alloc(few_ctx *c, size_t bytes, cudaStream_t st, void **out)
{
    *out = nullptr;
    if (bytes == 0) bytes = 256;
    bytes = align_up(bytes, 256);
    if (c->budget && c->in_use + bytes > c->budget) return FEW_ERR_BUDGET;
    cudaError_t e = cudaMallocFromPoolAsync(out, bytes, c->pool, st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *out = nullptr;
        return e == cudaErrorMemoryAllocation ? FEW_ERR_NOMEM : FEW_ERR_CUDA;
    }
    c->in_use += bytes;
    c->sizes[*out] = bytes;
    return FEW_OK;
}

void dev_free(few_ctx *c, void *p, cudaStream_t st)
{
    if (!p) return;
    auto it = c->sizes.find(p);
    if (it != c->sizes.end()) {
        c->in_use -= it->second;
        c->sizes.erase(it);
    }
    cudaFreeAsync(p, st);
}

// Event pair `slot` (0 build, 1 harmonics, 2 fold, 3 summation) around a kernel launch.
void tmark(few_ctx *c, int slot, bool end, cudaStream_t st)
{
    if (!c->timing) return;
    cudaEventRecord(c->tev[2 * slot + (end ? 1 : 0)], st);
    if (end) c->trec[slot] = true;
}

// Copy a host image to the device through a pinned staging block, ordered on `st`.
few_status upload(few_ctx *c, void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) return FEW_OK;
    PinnedPool::Block *b = c->pinned.acquire(bytes);
    if (!b) return FEW_ERR_NOMEM;
    std::memcpy(b->p, src, bytes);
    FEW_CUDA_TRY(cudaMemcpyAsync(dst, b->p, bytes, cudaMemcpyHostToDevice, st));
    FEW_CUDA_TRY(cudaEventRecord(b->ev, st));
    b->pending = true;
    return FEW_OK;
}

bool is_fin(double x) { return std::isfinite(x); }

few_status check_knots(const double *t, int K)
{
    if (!t || K < 4) return FEW_ERR_KNOTS;
    for (int k = 0; k < K; ++k)
        if (!is_fin(t[k])) return FEW_ERR_KNOTS;
    for (int k = 0; k + 1 < K; ++k)
        if (!(t[k + 1] > t[k])) return FEW_ERR_KNOTS;
    return FEW_OK;
}

// Harmonic slot plan of a mode list (host planning of the fold and the Horner order).
// Rows are the signed m from the largest down to m_last (-max m when any mode has m > 0, else
// 0), every m in between included; row j holds the slots n = hi_j, hi_j - 1, ..., lo_j (the
// extreme n of the signed modes with that m; zero-filled in between; an empty row has no slot
// and keeps the previous row's lo).  rows[j] = (slots of row j, lo_{j-1} - lo_j).
struct SlotPlan {
    int n_slots = 0, m_last = 0, lo_last = 0;
    std::vector<int2> pair_lm;
    std::vector<int> mode_pair;
    std::vector<int> slot_ptr;
    std::vector<int2> contrib;
    std::vector<int2> rows;
};

few_status plan_slots(const int *l, const int *m, const int *n, int N, SlotPlan &P)
{
    if (!l || !m || !n || N < 1) return FEW_ERR_MODES;
    std::set<std::tuple<int, int, int>> seen;
    int mmax = 0;
    for (int i = 0; i < N; ++i) {
        if (l[i] < 2 || l[i] > kMaxL || m[i] < 0 || m[i] > l[i] || n[i] < -kMaxAbsN ||
            n[i] > kMaxAbsN)
            return FEW_ERR_MODES;
        if (!seen.insert(std::make_tuple(l[i], m[i], n[i])).second) return FEW_ERR_MODES;
        mmax = std::max(mmax, m[i]);
    }
    // (l, m) pairs
    std::map<std::pair<int, int>, int> pairs;
    P.mode_pair.resize(N);
    for (int i = 0; i < N; ++i) {
        auto key = std::make_pair(l[i], m[i]);
        auto it = pairs.find(key);
        if (it == pairs.end()) {
            const int id = (int)P.pair_lm.size();
            pairs.emplace(key, id);
            P.pair_lm.push_back(make_int2(l[i], m[i]));
            P.mode_pair[i] = id;
        } else {
            P.mode_pair[i] = it->second;
        }
    }
    // n range of every signed m: the modes and, for m > 0, their (-m, -n) partners
    bool any_neg = false;
    for (int i = 0; i < N; ++i) any_neg |= (m[i] > 0);
    const int m_last = any_neg ? -mmax : 0;
    const int n_rows = mmax - m_last + 1;
    std::vector<int> lo(n_rows, kMaxAbsN + 1), hi(n_rows, -kMaxAbsN - 1);
    auto touch = [&](int ms, int ns) {
        const int j = mmax - ms;
        lo[j] = std::min(lo[j], ns);
        hi[j] = std::max(hi[j], ns);
    };
    for (int i = 0; i < N; ++i) {
        touch(m[i], n[i]);
        if (m[i] > 0) touch(-m[i], -n[i]);
    }
    // rows m = mmax..m_last, slots n = hi..lo in each
    std::map<std::pair<int, int>, int> slot_of;  // (signed m, n) -> slot
    int slot = 0, prev_lo = 0;
    for (int j = 0; j < n_rows; ++j) {
        const int ms = mmax - j;
        int L = 0, cur_lo = prev_lo;
        if (hi[j] >= lo[j]) {
            L = hi[j] - lo[j] + 1;
            cur_lo = lo[j];
            for (int q = hi[j]; q >= lo[j]; --q) slot_of[std::make_pair(ms, q)] = slot++;
        }
        P.rows.push_back(make_int2(L, j == 0 ? 0 : prev_lo - cur_lo));
        prev_lo = cur_lo;
    }
    P.n_slots = slot;
    P.m_last = m_last;
    P.lo_last = prev_lo;
    // contributions CSR
    std::vector<std::vector<int>> lists(slot);
    for (int i = 0; i < N; ++i) {
        lists[slot_of[std::make_pair(m[i], n[i])]].push_back(2 * i);
        if (m[i] > 0) lists[slot_of[std::make_pair(-m[i], -n[i])]].push_back(2 * i + 1);
    }
    P.slot_ptr.assign(slot + 1, 0);
    for (int s = 0; s < slot; ++s) P.slot_ptr[s + 1] = P.slot_ptr[s] + (int)lists[s].size();
    P.contrib.clear();
    P.contrib.reserve(P.slot_ptr[slot]);
    for (int s = 0; s < slot; ++s)
        for (int code : lists[s])
            P.contrib.push_back(make_int2(code, 2 * P.mode_pair[code >> 1] + (code & 1)));
    return FEW_OK;
}

few_status segments(const double *t, int K, double t0, double dt, int64_t ns, int64_t *seg)
{
    few_status st = check_knots(t, K);
    if (st) return st;
    if (!is_fin(t0) || !is_fin(dt) || !(dt > 0.0) || ns < 0 || ns > 2147483647LL) return FEW_ERR_RANGE;
    if (ns > 0) {
        const double last = std::fma((double)(ns - 1), dt, t0);
        if (t0 < t[0] || last > t[K - 1]) return FEW_ERR_RANGE;
    }
    seg[0] = 0;
    for (int k = 1; k < K - 1; ++k) {
        double x = std::ceil((t[k] - t0) / dt);
        int64_t v = x <= 0.0 ? 0 : (x >= (double)ns ? ns : (int64_t)x);
        seg[k] = std::max(v, seg[k - 1]);
    }
    seg[K - 1] = ns;
    return FEW_OK;
}

}  // namespace

struct few_traj {
    few_ctx *ctx = nullptr;
    int K = 0, N = 0, J = 0, S = 0;
    std::vector<double> t_host;
    SlotPlan plan;
    void *dmem = nullptr;
    double *ybuf = nullptr;  // device staging for host-provided knot data (lazy)
    BuildJob *job_dev = nullptr;
    TrajDev dev{};
    bool has_data = false;
    // device pointers of the current knot data (for batched rebuilds)
    const double *src_phi_phi = nullptr, *src_phi_r = nullptr, *src_re = nullptr, *src_im = nullptr;
};

struct few_batch {
    few_ctx *ctx = nullptr;
    bool fp64 = false;
    int variant = kVariantFp64;
    int n = 0;
    void *blob_dev = nullptr;
    void *scratch_dev = nullptr;
    void *jobs_dev = nullptr;
    int n_jobs = 0, build_blocks = 0, max_knots = 0;
    int grid = 0, threads = 0, R = 0, smem = 0, total_pairs = 0, total_fold = 0;
    int total_anchor_segs = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Host image of a plan (the blob) plus its scratch requirements.
struct PlanImage {
    std::vector<unsigned char> blob;
    size_t off_waves = 0, off_cta = 0, off_seg = 0, off_anc = 0;
    size_t scratch_bytes = 0;
    std::vector<size_t> fcoef_off, ylm_off, anchor_off;
    std::vector<std::vector<int64_t>> seg;  // per wave: segment sample ranges [K]
    bool fp64 = false;
    int variant = kVariantFp64;
    int grid = 0, threads = 0, R = 0, smem = 0, buf_bytes = 0, total_pairs = 0, total_fold = 0;
    int total_anchor_segs = 0, stage_slots = 0, ring = 0;
};

int occupancy(few_ctx *c, int variant, int R, int T, int smem)
{
    auto key = std::make_tuple(variant, R, T, smem);
    auto it = c->occ_cache.find(key);
    if (it != c->occ_cache.end()) return it->second;
    const int o = sum_occupancy(variant, R, T, smem);
    c->occ_cache[key] = o;
    return o;
}

few_status validate_request(const few_request &r, bool need_device_out)
{
    if (!r.traj || !r.out) return FEW_ERR_INVALID_ARG;
    if (!r.traj->has_data) return FEW_ERR_STATE;
    if (r.prec != FEW_FP64 && r.prec != FEW_MIXED) return FEW_ERR_INVALID_ARG;
    if (r.out_where != FEW_MEM_HOST && r.out_where != FEW_MEM_DEVICE) return FEW_ERR_INVALID_ARG;
    if (need_device_out && r.out_where != FEW_MEM_DEVICE) return FEW_ERR_INVALID_ARG;
    if (!is_fin(r.theta) || !is_fin(r.phi) || !is_fin(r.scale) || !is_fin(r.dphi_phi0) ||
        !is_fin(r.dphi_r0))
        return FEW_ERR_INVALID_ARG;
    if (r.frame != FEW_FRAME_SOURCE && r.frame != FEW_FRAME_SSB) return FEW_ERR_INVALID_ARG;
    if (r.frame == FEW_FRAME_SSB) {
        if (!is_fin(r.theta_K) || !is_fin(r.phi_K)) return FEW_ERR_INVALID_ARG;
        // the source frame needs R x S != 0
        const double R[3] = {std::sin(r.theta) * std::cos(r.phi), std::sin(r.theta) * std::sin(r.phi),
                             std::cos(r.theta)};
        const double S[3] = {std::sin(r.theta_K) * std::cos(r.phi_K),
                             std::sin(r.theta_K) * std::sin(r.phi_K), std::cos(r.theta_K)};
        const double x = R[1] * S[2] - R[2] * S[1], y = R[2] * S[0] - R[0] * S[2],
                     z = R[0] * S[1] - R[1] * S[0];
        if (!(x * x + y * y + z * z > 1e-24)) return FEW_ERR_INVALID_ARG;
    }
    if (!is_fin(r.t0) || !is_fin(r.dt) || !(r.dt > 0.0) || r.n_samples < 0 ||
        r.n_samples > 2147483647LL)
        return FEW_ERR_RANGE;
    const few_traj *tr = r.traj;
    if (r.n_samples > 0) {
        const double last = std::fma((double)(r.n_samples - 1), r.dt, r.t0);
        if (r.t0 < tr->t_host[0] || last > tr->t_host[tr->K - 1]) return FEW_ERR_RANGE;
    }
    return FEW_OK;
}

// Build the host image of a plan for `n` requests of one precision.
few_status build_image(few_ctx *c, const few_request *reqs, int n, PlanImage &P)
{
    P.fp64 = reqs[0].prec == FEW_FP64;
    const int pi = P.fp64 ? 0 : 1;
    P.R = c->tile_R[pi];
    P.threads = c->tile_T[pi];
    int max_slots = 1;
    for (int q = 0; q < n; ++q) max_slots = std::max(max_slots, reqs[q].traj->plan.n_slots);
    P.variant = P.fp64 ? kVariantFp64 : kVariantScalar;
    const size_t slot_bytes = (size_t)sum_slot_bytes(P.variant);
    P.stage_slots = std::min(c->tile_S[pi], max_slots);  // no stage larger than any table
    P.ring = kDefaultRing;
    P.buf_bytes = (int)align_up((size_t)P.stage_slots * slot_bytes, 128);
    P.smem = P.ring * P.buf_bytes;
    const int occ = occupancy(c, P.variant, P.R, P.threads, P.smem);
    if (occ <= 0) return FEW_ERR_LIMIT;
    P.grid = c->sm_count * occ;

    // layout of the blob
    size_t off = align_up(sizeof(PlanHdr), 64);
    P.off_waves = off;
    off = align_up(off + sizeof(WaveDev) * n, 64);
    P.off_cta = off;
    off = align_up(off + sizeof(CtaStart) * (P.grid + 1), 64);
    P.off_seg = off;
    size_t seg_ints = 0;
    for (int q = 0; q < n; ++q) seg_ints += reqs[q].traj->K;
    off = align_up(off + sizeof(int) * seg_ints, 64);
    P.off_anc = off;  // per wave: first anchor of each segment, then the wave's total
    if (!P.fp64) off += sizeof(int) * seg_ints;
    off = align_up(off, 256);
    P.blob.assign(off, 0);
    P.seg.resize(n);
    for (int q = 0; q < n; ++q) {
        const few_request &r = reqs[q];
        P.seg[q].resize(r.traj->K);
        segments(r.traj->t_host.data(), r.traj->K, r.t0, r.dt, r.n_samples, P.seg[q].data());
    }

    // scratch: folded coefficients and harmonic tables per wave
    size_t s_off = 0;
    P.fcoef_off.resize(n);
    P.ylm_off.resize(n);
    P.anchor_off.resize(n);
    for (int q = 0; q < n; ++q) {
        const few_traj *tr = reqs[q].traj;
        P.fcoef_off[q] = s_off;
        s_off = align_up(s_off + (size_t)tr->S * tr->plan.n_slots * slot_bytes, 256);
        P.ylm_off[q] = s_off;
        s_off = align_up(s_off + (size_t)tr->plan.pair_lm.size() * 2 * sizeof(double2), 256);
        P.anchor_off[q] = s_off;
        if (!P.fp64) {
            int na = 0;
            for (int k = 0; k + 1 < tr->K; ++k)
                na += anchors_in_segment((int)P.seg[q][k], (int)P.seg[q][k + 1]);
            s_off = align_up(s_off + sizeof(Anchor) * (size_t)na, 256);
        }
    }
    P.scratch_bytes = s_off;
    return FEW_OK;
}

// CTA slices of the concatenated (wave, sample) space of n waves (segs[q]: wave q's K[q]
// segment starts, the last its sample count), cut at pass boundaries.  A pass is `pass`
// consecutive samples of one segment, and it costs a full pass (one Horner step per slot plus the
// fixed phase work, for every thread) even when its segment ends early; so every slice gets an
// equal share of the total pass cost, to within one pass, rather than an equal share of the
// samples (which left some slices several short passes more than others).  cta[grid] = (n, 0).
void partition_ctas(int n, const int64_t *const *segs, const int *K, const int *slots, int grid,
                    long long pass, CtaStart *cta)
{
    std::vector<long double> cost(n), cum(n + 1, 0.0L);
    std::vector<long long> npass(n, 0);
    auto seg_passes = [&](int q, int k) { return (segs[q][k + 1] - segs[q][k] + pass - 1) / pass; };
    for (int q = 0; q < n; ++q) {
        for (int k = 0; k + 1 < K[q]; ++k) npass[q] += seg_passes(q, k);
        cost[q] = (long double)(slots[q] + 16);
        cum[q + 1] = cum[q] + (long double)npass[q] * cost[q];
    }
    const long double total = cum[n];
    int q = 0, sk = 0;
    long long before = 0;  // passes of wave q before its segment sk
    cta[grid] = CtaStart{n, 0};
    for (int g = 0; g < grid; ++g) {
        if (total <= 0.0L) {
            cta[g] = CtaStart{n, 0};
            continue;
        }
        const long double x = total * g / grid;
        while (q < n - 1 && cum[q + 1] <= x) {
            ++q;
            sk = 0;
            before = 0;
        }
        // first pass of wave q whose cost starts at or after x, then the segment holding it
        long long k = (long long)std::ceil((x - cum[q]) / cost[q]);
        k = std::max(0LL, std::min(k, npass[q]));
        const int S = K[q] - 1;
        while (sk < S && before + seg_passes(q, sk) <= k) {
            before += seg_passes(q, sk);
            ++sk;
        }
        const long long ns = segs[q][S];
        const long long sample = sk < S ? segs[q][sk] + (k - before) * pass : ns;
        cta[g] = CtaStart{q, (int)std::min<long long>(sample, ns)};
    }
}

// Fill the blob now that the device addresses of blob and scratch are known.
void fill_image(few_ctx *c, const few_request *reqs, int n, PlanImage &P, unsigned char *blob_dev,
                unsigned char *scratch_dev, void *const *outs)
{
    PlanHdr *hdr = reinterpret_cast<PlanHdr *>(P.blob.data());
    WaveDev *wv = reinterpret_cast<WaveDev *>(P.blob.data() + P.off_waves);
    CtaStart *cta = reinterpret_cast<CtaStart *>(P.blob.data() + P.off_cta);
    int *seg = reinterpret_cast<int *>(P.blob.data() + P.off_seg);
    int *anc = reinterpret_cast<int *>(P.blob.data() + P.off_anc);
    size_t seg_pos = 0;
    int pair_begin = 0, fold_begin = 0, anchor_seg_begin = 0;
    for (int q = 0; q < n; ++q) {
        const few_request &r = reqs[q];
        const few_traj *tr = r.traj;
        WaveDev &W = wv[q];
        std::memset(&W, 0, sizeof(W));
        W.tr = tr->dev;
        W.theta = r.theta;
        W.phi = r.phi;
        W.scale = r.scale;
        W.dphi_phi = r.dphi_phi0;
        W.dphi_r = r.dphi_r0;
        W.frame = r.frame;
        W.theta_K = r.theta_K;
        W.phi_K = r.phi_K;
        W.t0 = r.t0;
        W.dt = r.dt;
        W.n_samples = (int)r.n_samples;
        W.out_c64 = r.out_c64 ? 1 : 0;
        W.out = outs[q];
        W.fcoef = scratch_dev + P.fcoef_off[q];
        W.ylm = reinterpret_cast<double2 *>(scratch_dev + P.ylm_off[q]);
        const std::vector<int64_t> &ss = P.seg[q];
        for (int k = 0; k < tr->K; ++k) seg[seg_pos + k] = (int)ss[k];
        W.seg_start = reinterpret_cast<const int *>(blob_dev + P.off_seg) + seg_pos;
        if (!P.fp64) {
            int a = 0;
            for (int k = 0; k + 1 < tr->K; ++k) {
                anc[seg_pos + k] = a;
                a += anchors_in_segment((int)ss[k], (int)ss[k + 1]);
            }
            anc[seg_pos + tr->K - 1] = a;
            W.anchors = reinterpret_cast<Anchor *>(scratch_dev + P.anchor_off[q]);
            W.anchor_off = reinterpret_cast<const int *>(blob_dev + P.off_anc) + seg_pos;
            W.anchor_seg_begin = anchor_seg_begin;
            anchor_seg_begin += tr->S;
        }
        seg_pos += tr->K;
        W.pair_begin = pair_begin;
        pair_begin += (int)tr->plan.pair_lm.size();
        W.fold_blocks_per_seg = (tr->plan.n_slots + kFoldThreads - 1) / kFoldThreads;
        W.fold_begin = fold_begin;
        fold_begin += tr->S * W.fold_blocks_per_seg;
    }
    P.total_pairs = pair_begin;
    P.total_fold = fold_begin;
    P.total_anchor_segs = anchor_seg_begin;
    {
        std::vector<const int64_t *> segs(n);
        std::vector<int> Ks(n), slots(n);
        for (int q = 0; q < n; ++q) {
            segs[q] = P.seg[q].data();
            Ks[q] = reqs[q].traj->K;
            slots[q] = reqs[q].traj->plan.n_slots;
        }
        partition_ctas(n, segs.data(), Ks.data(), slots.data(), P.grid,
                       (long long)P.threads * P.R, cta);
    }
    hdr->n_waves = n;
    hdr->total_pairs = P.total_pairs;
    hdr->total_fold_blocks = P.total_fold;
    hdr->total_anchor_segs = P.total_anchor_segs;
    hdr->grid_sum = P.grid;
    hdr->buf_bytes = P.buf_bytes;
    hdr->stage_slots = P.stage_slots;
    hdr->ring = P.ring;
    hdr->variant = P.variant;
    hdr->waves = reinterpret_cast<const WaveDev *>(blob_dev + P.off_waves);
    hdr->cta = reinterpret_cast<const CtaStart *>(blob_dev + P.off_cta);
    hdr->err = c->d_err;
}

few_status launch_kernels(few_ctx *c, const PlanHdr *hdr_dev, int total_pairs, int total_fold,
                          int total_anchor_segs, int grid, int threads, int R, int smem, int variant,
                          cudaStream_t st)
{
    // the phase anchors depend on the splines only: they run on a side lane beside the
    // harmonics and the fold (FP64-pipe work next to latency-bound work), joined before the sum
    const bool fork = total_anchor_segs > 0;
    auto &L = c->lanes[c->lane_next++ % 4];
    if (fork) {
        // any failure after this point still leaves the side stream's work ordered before what
        // the caller queues next on `st` (the release of the call's scratch)
        if (cudaEventRecord(L.fork, st) != cudaSuccess ||
            cudaStreamWaitEvent(L.s, L.fork, 0) != cudaSuccess)
            return FEW_ERR_CUDA;
        const cudaError_t ea = launch_anchor(hdr_dev, total_anchor_segs, L.s);
        if (cudaEventRecord(L.join, L.s) != cudaSuccess) {
            cudaStreamSynchronize(L.s);
            return FEW_ERR_CUDA;
        }
        if (ea != cudaSuccess) {
            cudaStreamWaitEvent(st, L.join, 0);
            return FEW_ERR_CUDA;
        }
    }
    auto joined = [&](cudaError_t e) {  // a failed launch: join the side stream, then report
        if (e == cudaSuccess) return true;
        if (fork) cudaStreamWaitEvent(st, L.join, 0);
        return false;
    };
    tmark(c, 1, false, st);
    if (!joined(launch_ylm(hdr_dev, total_pairs, variant == kVariantFp64, st))) return FEW_ERR_CUDA;
    tmark(c, 1, true, st);
    tmark(c, 2, false, st);
    if (!joined(launch_fold(hdr_dev, total_fold, variant == kVariantFp64, st))) return FEW_ERR_CUDA;
    if (fork) FEW_CUDA_TRY(cudaStreamWaitEvent(st, L.join, 0));
    tmark(c, 2, true, st);
    tmark(c, 3, false, st);
    FEW_CUDA_TRY(launch_sum(hdr_dev, grid, threads, R, smem, variant, st));
    tmark(c, 3, true, st);
    return FEW_OK;
}

const char *kNames[] = {"FEW_OK",           "FEW_ERR_INVALID_ARG", "FEW_ERR_KNOTS",
                        "FEW_ERR_MODES",    "FEW_ERR_RANGE",       "FEW_ERR_NOMEM",
                        "FEW_ERR_BUDGET",   "FEW_ERR_CUDA",        "FEW_ERR_TIMEOUT",
                        "FEW_ERR_LIMIT",    "FEW_ERR_STATE"};

}  // namespace

// ------------------------------------------------------------------------------ C ABI

extern "C" {

const char *few_strerror(few_status s)
{
    const int i = (int)s;
    if (i < 0 || i >= (int)(sizeof(kNames) / sizeof(kNames[0]))) return "FEW_ERR_UNKNOWN";
    return kNames[i];
}

int few_abi_version(void) { return FEW_ABI_VERSION; }

few_status few_ctx_create(few_ctx **out, int device, size_t hbm_budget_bytes)
{
    if (!out) return FEW_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        (void)cudaGetLastError();
        return FEW_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return FEW_ERR_INVALID_ARG;
    few_ctx *c = new (std::nothrow) few_ctx();
    if (!c) return FEW_ERR_NOMEM;
    c->device = device;
    c->budget = hbm_budget_bytes;
    auto fail = [&](few_status s) {
        if (c->d_err) cudaFree(c->d_err);
        if (c->internal) cudaStreamDestroy(c->internal);
        for (auto &l : c->lanes) {
            if (l.s) cudaStreamDestroy(l.s);
            if (l.fork) cudaEventDestroy(l.fork);
            if (l.join) cudaEventDestroy(l.join);
        }
        for (auto &e : c->tev)
            if (e) cudaEventDestroy(e);
        if (c->pool) cudaMemPoolDestroy(c->pool);
        (void)cudaGetLastError();
        delete c;
        return s;
    };
    DeviceScope dev_scope(device);
    if (!dev_scope.ok) return fail(FEW_ERR_CUDA);
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return fail(FEW_ERR_CUDA);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess) return fail(FEW_ERR_CUDA);
    uint64_t thresh = UINT64_MAX;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thresh);
    if (cudaStreamCreateWithFlags(&c->internal, cudaStreamNonBlocking) != cudaSuccess)
        return fail(FEW_ERR_CUDA);
    for (auto &l : c->lanes)
        if (cudaStreamCreateWithFlags(&l.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&l.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&l.join, cudaEventDisableTiming) != cudaSuccess)
            return fail(FEW_ERR_CUDA);
    if (cudaMalloc(&c->d_err, sizeof(unsigned)) != cudaSuccess) return fail(FEW_ERR_NOMEM);
    if (cudaMemset(c->d_err, 0, sizeof(unsigned)) != cudaSuccess) return fail(FEW_ERR_CUDA);
    if (sum_configure() != cudaSuccess) return fail(FEW_ERR_CUDA);
    for (auto &e : c->tev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(FEW_ERR_CUDA);
    *out = c;
    return FEW_OK;
}

few_status few_batch_release(few_ctx *ctx, few_batch *b);
few_status few_traj_release(few_ctx *ctx, few_traj *t);
few_status few_basis_release(few_ctx *ctx, few_basis *b);

few_status few_ctx_destroy(few_ctx *ctx)
{
    if (!ctx) return FEW_OK;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        DeviceScope dev_scope(ctx->device);
        cudaDeviceSynchronize();
        auto bs = ctx->batches;
        for (few_batch *b : bs) few_batch_release(ctx, b);
        auto ts = ctx->trajs;
        for (few_traj *t : ts) few_traj_release(ctx, t);
        auto rbs = ctx->bases;
        for (few_basis *b : rbs) few_basis_release(ctx, b);
        cudaStreamSynchronize(ctx->internal);
        for (auto &e : ctx->tev)
            if (e) cudaEventDestroy(e);
        ctx->pinned.release();
        cudaFree(ctx->d_err);
        cudaStreamDestroy(ctx->internal);
        for (auto &l : ctx->lanes) {
            cudaStreamDestroy(l.s);
            cudaEventDestroy(l.fork);
            cudaEventDestroy(l.join);
        }
        cudaMemPoolDestroy(ctx->pool);
        (void)cudaGetLastError();
    }
    delete ctx;
    return FEW_OK;
}

few_status few_ctx_memory(few_ctx *ctx, size_t *bytes_in_use, size_t *budget_bytes)
{
    if (!ctx) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (bytes_in_use) *bytes_in_use = ctx->in_use;
    if (budget_bytes) *budget_bytes = ctx->budget;
    return FEW_OK;
}

few_status few_traj_create(few_ctx *ctx, const double *t_knots, int K, const int *l, const int *m,
                           const int *n, int N, few_traj **out)
{
    NvtxRange nvtx_range("few_traj_create");
    if (!ctx || !out) return FEW_ERR_INVALID_ARG;
    *out = nullptr;
    few_status st = check_knots(t_knots, K);
    if (st) return st;
    if (K > FEW_MAX_KNOTS) return FEW_ERR_LIMIT;
    SlotPlan plan;
    if ((st = plan_slots(l, m, n, N, plan))) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    few_traj *tr = new (std::nothrow) few_traj();
    if (!tr) return FEW_ERR_NOMEM;
    tr->ctx = ctx;
    tr->K = K;
    tr->N = N;
    tr->J = 2 + 2 * N;
    tr->S = K - 1;
    tr->t_host.assign(t_knots, t_knots + K);
    tr->plan = std::move(plan);
    const SlotPlan &P = tr->plan;

    // one device allocation for every trajectory array
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_t = take(sizeof(double) * K), o_h = take(sizeof(double) * K),
                 o_ih = take(sizeof(double) * K), o_ra = take(sizeof(double) * K),
                 o_rb = take(sizeof(double) * K), o_lo = take(sizeof(double) * K),
                 o_up = take(sizeof(double) * K),
                 o_ip = take(sizeof(double) * K), o_v = take(sizeof(double) * K),
                 o_x = take(sizeof(double) * K),
                 o_sinv = take(sizeof(double) * (kBuildParts - 1) * (kBuildParts - 1)),
                 o_parts = take(sizeof(int) * (kBuildParts + 2)),
                 o_coef = take(sizeof(double) * 4 * (size_t)tr->S * tr->J),
                 o_slopes = take(sizeof(double) * (size_t)K * tr->J),
                 o_pair = take(sizeof(int2) * P.pair_lm.size()), o_mp = take(sizeof(int) * N),
                 o_sp = take(sizeof(int) * P.slot_ptr.size()),
                 o_ct = take(sizeof(int2) * std::max<size_t>(1, P.contrib.size())),
                 o_rows = take(sizeof(int2) * P.rows.size()), o_job = take(sizeof(BuildJob));
    if ((st = dev_alloc(ctx, off, ctx->internal, &tr->dmem))) {
        delete tr;
        return st;
    }
    unsigned char *d = static_cast<unsigned char *>(tr->dmem);
    // host image of the small arrays
    std::vector<unsigned char> img(o_coef, 0);
    std::memcpy(img.data() + o_t, t_knots, sizeof(double) * K);
    std::vector<unsigned char> img2(off - o_pair, 0);
    auto put = [&](size_t o, const void *src, size_t bytes) {
        if (bytes) std::memcpy(img2.data() + (o - o_pair), src, bytes);
    };
    put(o_pair, P.pair_lm.data(), sizeof(int2) * P.pair_lm.size());
    put(o_mp, P.mode_pair.data(), sizeof(int) * N);
    put(o_sp, P.slot_ptr.data(), sizeof(int) * P.slot_ptr.size());
    put(o_ct, P.contrib.data(), sizeof(int2) * P.contrib.size());
    put(o_rows, P.rows.data(), sizeof(int2) * P.rows.size());

    TrajDev &D = tr->dev;
    D.K = K;
    D.N = N;
    D.J = tr->J;
    D.S = tr->S;
    D.n_pairs = (int)P.pair_lm.size();
    D.n_slots = P.n_slots;
    D.n_rows = (int)P.rows.size();
    D.m_last = P.m_last;
    D.lo_last = P.lo_last;
    D.t = reinterpret_cast<const double *>(d + o_t);
    D.h = reinterpret_cast<const double *>(d + o_h);
    D.inv_h = reinterpret_cast<const double *>(d + o_ih);
    D.fac_ra = reinterpret_cast<const double *>(d + o_ra);
    D.fac_rb = reinterpret_cast<const double *>(d + o_rb);
    D.fac_lo = reinterpret_cast<const double *>(d + o_lo);
    D.fac_up = reinterpret_cast<const double *>(d + o_up);
    D.fac_ip = reinterpret_cast<const double *>(d + o_ip);
    D.fac_v = reinterpret_cast<const double *>(d + o_v);
    D.fac_x = reinterpret_cast<const double *>(d + o_x);
    D.fac_sinv = reinterpret_cast<const double *>(d + o_sinv);
    D.parts = reinterpret_cast<const int *>(d + o_parts);
    D.coef = reinterpret_cast<double *>(d + o_coef);
    D.slopes = reinterpret_cast<double *>(d + o_slopes);
    D.pair_lm = reinterpret_cast<const int2 *>(d + o_pair);
    D.mode_pair = reinterpret_cast<const int *>(d + o_mp);
    D.slot_ptr = reinterpret_cast<const int *>(d + o_sp);
    D.contrib = reinterpret_cast<const int2 *>(d + o_ct);
    D.rows = reinterpret_cast<const int2 *>(d + o_rows);
    tr->job_dev = reinterpret_cast<BuildJob *>(d + o_job);

    cudaStream_t s = ctx->internal;
    few_status us = upload(ctx, d, img.data(), o_h, s);  // knot times
    if (!us) us = upload(ctx, d + o_pair, img2.data(), off - o_pair, s);
    cudaError_t e = cudaSuccess;
    if (!us) {
        FactorArrays fa;
        fa.h = reinterpret_cast<double *>(d + o_h);
        fa.inv_h = reinterpret_cast<double *>(d + o_ih);
        fa.ra = reinterpret_cast<double *>(d + o_ra);
        fa.rb = reinterpret_cast<double *>(d + o_rb);
        fa.lo = reinterpret_cast<double *>(d + o_lo);
        fa.up = reinterpret_cast<double *>(d + o_up);
        fa.ip = reinterpret_cast<double *>(d + o_ip);
        fa.v = reinterpret_cast<double *>(d + o_v);
        fa.x = reinterpret_cast<double *>(d + o_x);
        fa.sinv = reinterpret_cast<double *>(d + o_sinv);
        fa.parts = reinterpret_cast<int *>(d + o_parts);
        e = launch_factor(D.t, K, fa, s);
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (us || e != cudaSuccess || e2 != cudaSuccess) {
        (void)cudaGetLastError();
        dev_free(ctx, tr->dmem, s);
        cudaStreamSynchronize(s);
        delete tr;
        return us ? us : FEW_ERR_CUDA;
    }
    ctx->trajs.insert(tr);
    *out = tr;
    return FEW_OK;
}

few_status few_traj_set_data(few_ctx *ctx, few_traj *tr, const double *phi_phi, const double *phi_r,
                             const double *amp_re, const double *amp_im, few_mem where, void *stream)
{
    NvtxRange nvtx_range("few_traj_set_data");
    if (!ctx || !tr || tr->ctx != ctx) return FEW_ERR_INVALID_ARG;
    if (!phi_phi || !phi_r || !amp_re || !amp_im) return FEW_ERR_INVALID_ARG;
    if (where != FEW_MEM_HOST && where != FEW_MEM_DEVICE) return FEW_ERR_INVALID_ARG;
    std::unique_lock<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t K = tr->K, N = tr->N;
    BuildJob job{};
    job.tr = tr->dev;
    cudaEvent_t copied = nullptr;  // host inputs: completion of their copies
    if (where == FEW_MEM_HOST) {
        if (!tr->ybuf) {
            void *p = nullptr;
            few_status s = dev_alloc(ctx, sizeof(double) * (2 * K + 2 * K * N), ctx->internal, &p);
            if (s) return s;
            if (cudaStreamSynchronize(ctx->internal) != cudaSuccess) return FEW_ERR_CUDA;
            tr->ybuf = static_cast<double *>(p);
        }
        double *y = tr->ybuf;
        FEW_CUDA_TRY(cudaMemcpyAsync(y, phi_phi, sizeof(double) * K, cudaMemcpyHostToDevice, st));
        FEW_CUDA_TRY(cudaMemcpyAsync(y + K, phi_r, sizeof(double) * K, cudaMemcpyHostToDevice, st));
        FEW_CUDA_TRY(cudaMemcpyAsync(y + 2 * K, amp_re, sizeof(double) * K * N, cudaMemcpyHostToDevice, st));
        FEW_CUDA_TRY(cudaMemcpyAsync(y + 2 * K + K * N, amp_im, sizeof(double) * K * N,
                                     cudaMemcpyHostToDevice, st));
        // the caller may reuse its host arrays on return: the copies' completion is waited for
        // after the build is queued behind them, so the device does not idle on the host
        FEW_CUDA_TRY(cudaEventCreateWithFlags(&copied, cudaEventDisableTiming));
        if (cudaEventRecord(copied, st) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaEventDestroy(copied);
            return FEW_ERR_CUDA;
        }
        job.phi_phi = y;
        job.phi_r = y + K;
        job.amp_re = y + 2 * K;
        job.amp_im = y + 2 * K + K * N;
    } else {
        job.phi_phi = phi_phi;
        job.phi_r = phi_r;
        job.amp_re = amp_re;
        job.amp_im = amp_im;
    }
    job.block_begin = 0;
    few_status s = upload(ctx, tr->job_dev, &job, sizeof(job), st);
    const int blocks = (tr->J + kBuildSplines - 1) / kBuildSplines;
    if (!s) {
        tmark(ctx, 0, false, st);
        if (launch_build(tr->job_dev, 1, blocks, tr->K, ctx->d_err, st) != cudaSuccess) {
            (void)cudaGetLastError();
            s = FEW_ERR_CUDA;
        }
        tmark(ctx, 0, true, st);
    }
    if (copied) {
        lk.unlock();  // the copies' completion concerns this call only
        if (cudaEventSynchronize(copied) != cudaSuccess && !s) {
            (void)cudaGetLastError();
            s = FEW_ERR_CUDA;
        }
        cudaEventDestroy(copied);
    }
    if (s) return s;
    tr->src_phi_phi = job.phi_phi;
    tr->src_phi_r = job.phi_r;
    tr->src_re = job.amp_re;
    tr->src_im = job.amp_im;
    tr->has_data = true;
    return FEW_OK;
}

few_status few_traj_release(few_ctx *ctx, few_traj *tr)
{
    if (!ctx || !tr || tr->ctx != ctx) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    cudaDeviceSynchronize();
    dev_free(ctx, tr->ybuf, ctx->internal);
    dev_free(ctx, tr->dmem, ctx->internal);
    cudaStreamSynchronize(ctx->internal);
    (void)cudaGetLastError();
    ctx->trajs.erase(tr);
    delete tr;
    return FEW_OK;
}

few_status few_traj_info(const few_traj *tr, int *K, int *N, int *n_slots)
{
    if (!tr) return FEW_ERR_INVALID_ARG;
    if (K) *K = tr->K;
    if (N) *N = tr->N;
    if (n_slots) *n_slots = tr->plan.n_slots;
    return FEW_OK;
}

few_status few_waveform(few_ctx *ctx, const few_request *req, void *stream)
{
    NvtxRange nvtx_range("few_waveform");
    if (!ctx || !req) return FEW_ERR_INVALID_ARG;
    few_status st = validate_request(*req, false);
    if (st) return st;
    if (req->traj->ctx != ctx) return FEW_ERR_INVALID_ARG;
    if (req->n_samples == 0) return FEW_OK;
    std::unique_lock<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PlanImage P;
    if ((st = build_image(ctx, req, 1, P))) return st;
    const size_t out_bytes = (size_t)req->n_samples * (req->out_c64 ? 8 : 16);
    void *blob = nullptr, *scratch = nullptr, *dout = nullptr;
    if ((st = dev_alloc(ctx, P.blob.size(), s, &blob))) return st;
    if ((st = dev_alloc(ctx, P.scratch_bytes, s, &scratch))) {
        dev_free(ctx, blob, s);
        return st;
    }
    void *out_dev = req->out;
    if (req->out_where == FEW_MEM_HOST) {
        // page-locked host memory is addressable from the device (over NVLink-C2C on a Grace
        // host): the summation kernel stores into it directly and the transfer overlaps the
        // compute; pageable memory is staged on the device and copied back
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, req->out) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer != nullptr) {
            out_dev = pa.devicePointer;
        } else {
            (void)cudaGetLastError();
            if ((st = dev_alloc(ctx, out_bytes, s, &dout))) {
                dev_free(ctx, scratch, s);
                dev_free(ctx, blob, s);
                return st;
            }
            out_dev = dout;
        }
    }
    fill_image(ctx, req, 1, P, static_cast<unsigned char *>(blob),
               static_cast<unsigned char *>(scratch), &out_dev);
    st = upload(ctx, blob, P.blob.data(), P.blob.size(), s);
    if (!st)
        st = launch_kernels(ctx, static_cast<const PlanHdr *>(blob), P.total_pairs, P.total_fold,
                            P.total_anchor_segs, P.grid, P.threads, P.R, P.smem, P.variant, s);
    if (!st && dout) {
        cudaError_t e = cudaMemcpyAsync(req->out, dout, out_bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            st = FEW_ERR_CUDA;
        }
    }
    dev_free(ctx, dout, s);
    dev_free(ctx, scratch, s);
    dev_free(ctx, blob, s);
    if (!st && req->out_where == FEW_MEM_HOST) {
        // everything is queued: wait for the result without holding the context, so calls from
        // other host threads (their own streams) overlap this one's transfer and compute
        lk.unlock();
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            (void)cudaGetLastError();
            st = FEW_ERR_CUDA;
        }
    }
    return st;
}

few_status few_phase_samples(few_ctx *ctx, const few_traj *tr, double t0, double dt, int64_t n,
                             double dphi_phi0, double dphi_r0, double *out_dev, void *stream)
{
    NvtxRange nvtx_range("few_phase_samples");
    if (!ctx || !tr || tr->ctx != ctx || !out_dev) return FEW_ERR_INVALID_ARG;
    if (!tr->has_data) return FEW_ERR_STATE;
    if (!is_fin(dphi_phi0) || !is_fin(dphi_r0)) return FEW_ERR_INVALID_ARG;
    std::vector<int64_t> seg(tr->K);
    few_status st = segments(tr->t_host.data(), tr->K, t0, dt, n, seg.data());
    if (st) return st;
    if (n == 0) return FEW_OK;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int> seg32(seg.begin(), seg.end());
    void *d = nullptr;
    if ((st = dev_alloc(ctx, sizeof(int) * seg32.size(), s, &d))) return st;
    st = upload(ctx, d, seg32.data(), sizeof(int) * seg32.size(), s);
    if (!st) {
        cudaError_t e = launch_phases(tr->dev, static_cast<const int *>(d), t0, dt, (int)n,
                                      dphi_phi0, dphi_r0, out_dev, s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            st = FEW_ERR_CUDA;
        }
    }
    dev_free(ctx, d, s);
    return st;
}

few_status few_mode_select(few_ctx *ctx, const double *amp_re, const double *amp_im, int K, int N,
                           const int *m, double eps, unsigned char *mask, void *stream)
{
    NvtxRange nvtx_range("few_mode_select");
    if (!ctx || !amp_re || !amp_im || !m || !mask) return FEW_ERR_INVALID_ARG;
    if (K < 1 || N < 1 || !is_fin(eps) || eps < 0.0) return FEW_ERR_INVALID_ARG;
    if (N > mode_select_max_modes()) return FEW_ERR_LIMIT;
    ModeDoubling dbl{};
    for (int i = 0; i < N; ++i) {
        if (m[i] < 0) return FEW_ERR_MODES;
        if (m[i] > 0) dbl.w[i >> 5] |= 1u << (i & 31);
    }
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (launch_mode_select(amp_re, amp_im, K, N, dbl, eps, mask, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return FEW_ERR_CUDA;
    }
    return FEW_OK;
}

few_status few_direct_sum(few_ctx *ctx, const double *pphi, const double *pr, const double *are,
                          const double *aim, int64_t ns, const int *l, const int *m, const int *n,
                          int N, double theta, double phi, double scale, int prec, void *out,
                          int out_c64, void *stream)
{
    NvtxRange nvtx_range("few_direct_sum");
    if (!ctx || !pphi || !pr || !are || !aim || !out) return FEW_ERR_INVALID_ARG;
    if (prec != FEW_FP64 && prec != FEW_MIXED) return FEW_ERR_INVALID_ARG;
    if (!is_fin(theta) || !is_fin(phi) || !is_fin(scale) || ns < 0) return FEW_ERR_INVALID_ARG;
    SlotPlan P;
    few_status st = plan_slots(l, m, n, N, P);  // validates the modes
    if (st) return st;
    if (ns == 0) return FEW_OK;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t mc_bytes = align_up(direct_mode_const_bytes(N), 256);
    const size_t idx_bytes = align_up(sizeof(int) * (size_t)N, 256);
    void *d = nullptr;
    if ((st = dev_alloc(ctx, mc_bytes + 3 * idx_bytes, s, &d))) return st;
    unsigned char *b = static_cast<unsigned char *>(d);
    std::vector<int> lmn(3 * (idx_bytes / sizeof(int)), 0);
    const size_t stride = idx_bytes / sizeof(int);
    std::copy(l, l + N, lmn.begin());
    std::copy(m, m + N, lmn.begin() + stride);
    std::copy(n, n + N, lmn.begin() + 2 * stride);
    st = upload(ctx, b + mc_bytes, lmn.data(), 3 * idx_bytes, s);
    if (!st) {
        const int *dl = reinterpret_cast<const int *>(b + mc_bytes);
        cudaError_t e = launch_direct(pphi, pr, are, aim, (long long)ns, dl, dl + stride,
                                      dl + 2 * stride, N, theta, phi, scale, prec == FEW_FP64, out,
                                      out_c64 ? 1 : 0, b, ctx->sm_count, s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            st = FEW_ERR_CUDA;
        }
    }
    dev_free(ctx, d, s);
    return st;
}

// Reduced basis (Sec. 3.E): FP64 B, its transposed Gram matrix in FP64 and FP32, and the split
// bf16 operand of the tensor-core product, in one device allocation.
struct few_basis {
    few_ctx *ctx = nullptr;
    int Nb = 0, N = 0;
    void *dmem = nullptr;
    const double *bre = nullptr, *bim = nullptr;
    const double2 *gt64 = nullptr;
    const float2 *gt32 = nullptr;
    const int *bexp = nullptr;
    const unsigned char *bpack = nullptr;
};

few_status few_basis_create(few_ctx *ctx, const double *b_re, const double *b_im, int Nb, int N,
                            few_mem where, void *stream, few_basis **out)
{
    NvtxRange nvtx_range("few_basis_create");
    if (!ctx || !b_re || !b_im || !out || Nb < 1 || N < 1) return FEW_ERR_INVALID_ARG;
    if (where != FEW_MEM_HOST && where != FEW_MEM_DEVICE) return FEW_ERR_INVALID_ARG;
    if (Nb > FEW_MAX_BASIS) return FEW_ERR_LIMIT;
    *out = nullptr;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const RbLayout L = rb_layout(Nb, N, 0);
    const size_t b_bytes = align_up(sizeof(double) * (size_t)Nb * N, 256);
    const size_t g64 = align_up(sizeof(double2) * (size_t)Nb * Nb, 256);
    const size_t g32 = align_up(sizeof(float2) * (size_t)Nb * Nb, 256);
    const size_t ex = align_up(sizeof(int) * (size_t)L.modes_padded, 256);
    void *d = nullptr;
    few_status st = dev_alloc(ctx, 2 * b_bytes + g64 + g32 + ex + L.bpack_bytes, s, &d);
    if (st) return st;
    unsigned char *p = static_cast<unsigned char *>(d);
    double *bre = reinterpret_cast<double *>(p), *bim = reinterpret_cast<double *>(p + b_bytes);
    const size_t bytes = sizeof(double) * (size_t)Nb * N;
    if (where == FEW_MEM_HOST) {
        st = upload(ctx, bre, b_re, bytes, s);
        if (!st) st = upload(ctx, bim, b_im, bytes, s);
    } else if (cudaMemcpyAsync(bre, b_re, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
               cudaMemcpyAsync(bim, b_im, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        (void)cudaGetLastError();
        st = FEW_ERR_CUDA;
    }
    auto *gt64 = reinterpret_cast<double2 *>(p + 2 * b_bytes);
    auto *gt32 = reinterpret_cast<float2 *>(p + 2 * b_bytes + g64);
    int *bexp = reinterpret_cast<int *>(p + 2 * b_bytes + g64 + g32);
    unsigned char *bpack = p + 2 * b_bytes + g64 + g32 + ex;
    if (!st && launch_rb_basis(bre, bim, Nb, N, gt64, gt32, bexp, bpack, ctx->sm_count, s) != cudaSuccess) {
        (void)cudaGetLastError();
        st = FEW_ERR_CUDA;
    }
    if (st) {
        dev_free(ctx, d, s);
        return st;
    }
    auto *b = new few_basis;
    b->ctx = ctx;
    b->Nb = Nb;
    b->N = N;
    b->dmem = d;
    b->bre = bre;
    b->bim = bim;
    b->gt64 = gt64;
    b->gt32 = gt32;
    b->bexp = bexp;
    b->bpack = bpack;
    ctx->bases.insert(b);
    *out = b;
    return FEW_OK;
}

few_status few_basis_release(few_ctx *ctx, few_basis *b)
{
    if (!ctx || !b || b->ctx != ctx) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    cudaDeviceSynchronize();
    dev_free(ctx, b->dmem, ctx->internal);
    cudaStreamSynchronize(ctx->internal);
    (void)cudaGetLastError();
    ctx->bases.erase(b);
    delete b;
    return FEW_OK;
}

few_status few_rb_amplitudes(few_ctx *ctx, const few_basis *b, const double *are,
                             const double *aim, int M, const double *nu, int prec, double *ore,
                             double *oim, void *stream)
{
    NvtxRange nvtx_range("few_rb_amplitudes");
    if (!ctx || !b || b->ctx != ctx || M < 0) return FEW_ERR_INVALID_ARG;
    if (prec != FEW_FP64 && prec != FEW_MIXED) return FEW_ERR_INVALID_ARG;
    if (M == 0) return FEW_OK;
    if (!are || !aim || !ore || !oim) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool fp64 = prec == FEW_FP64;
    const RbLayout L = rb_layout(b->Nb, b->N, M);
    const size_t sc_bytes = align_up(2 * sizeof(double) * (size_t)M, 256);  // scale, then q
    const size_t ex_bytes = fp64 ? 0 : align_up(sizeof(int) * (size_t)L.rows_padded, 256);
    void *d = nullptr;
    few_status st = dev_alloc(ctx, sc_bytes + ex_bytes + (fp64 ? 0 : L.apack_bytes), s, &d);
    if (st) return st;
    unsigned char *p = static_cast<unsigned char *>(d);
    auto &lane = ctx->lanes[ctx->lane_next++ % 4];
    cudaError_t e = launch_rb(are, aim, M, b->Nb, b->N, nu, fp64, b->bre, b->bim, b->gt64, b->gt32,
                              b->bexp, b->bpack, reinterpret_cast<double *>(p),
                              reinterpret_cast<int *>(p + sc_bytes), p + sc_bytes + ex_bytes, ore,
                              oim, ctx->d_err, ctx->sm_count, s, lane.s, lane.fork, lane.join);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        st = FEW_ERR_CUDA;
    }
    dev_free(ctx, d, s);
    return st;
}

few_status few_batch_plan(few_ctx *ctx, const few_request *reqs, int n, unsigned flags, few_batch **out)
{
    NvtxRange nvtx_range("few_batch_plan");
    if (!ctx || !reqs || n < 1 || !out) return FEW_ERR_INVALID_ARG;
    *out = nullptr;
    for (int q = 0; q < n; ++q) {
        few_status st = validate_request(reqs[q], true);
        if (st) return st;
        if (reqs[q].traj->ctx != ctx || reqs[q].prec != reqs[0].prec) return FEW_ERR_INVALID_ARG;
    }
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    PlanImage P;
    few_status st = build_image(ctx, reqs, n, P);
    if (st) return st;
    few_batch *b = new (std::nothrow) few_batch();
    if (!b) return FEW_ERR_NOMEM;
    b->ctx = ctx;
    b->fp64 = P.fp64;
    b->variant = P.variant;
    b->n = n;
    cudaStream_t s = ctx->internal;
    auto fail = [&](few_status e) {
        dev_free(ctx, b->jobs_dev, s);
        dev_free(ctx, b->scratch_dev, s);
        dev_free(ctx, b->blob_dev, s);
        cudaStreamSynchronize(s);
        (void)cudaGetLastError();
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return e;
    };
    if ((st = dev_alloc(ctx, P.blob.size(), s, &b->blob_dev))) return fail(st);
    if ((st = dev_alloc(ctx, P.scratch_bytes, s, &b->scratch_dev))) return fail(st);
    std::vector<void *> outs(n);
    for (int q = 0; q < n; ++q) outs[q] = reqs[q].out;
    fill_image(ctx, reqs, n, P, static_cast<unsigned char *>(b->blob_dev),
               static_cast<unsigned char *>(b->scratch_dev), outs.data());
    if ((st = upload(ctx, b->blob_dev, P.blob.data(), P.blob.size(), s))) return fail(st);
    if (flags & FEW_BATCH_REBUILD_SPLINES) {
        std::vector<BuildJob> jobs;
        std::set<const few_traj *> seen;
        int blocks = 0;
        for (int q = 0; q < n; ++q) {
            const few_traj *tr = reqs[q].traj;
            if (!seen.insert(tr).second) continue;
            BuildJob j{};
            j.tr = tr->dev;
            j.phi_phi = tr->src_phi_phi;
            j.phi_r = tr->src_phi_r;
            j.amp_re = tr->src_re;
            j.amp_im = tr->src_im;
            j.block_begin = blocks;
            blocks += (tr->J + kBuildSplines - 1) / kBuildSplines;
            b->max_knots = std::max(b->max_knots, tr->K);
            jobs.push_back(j);
        }
        if ((st = dev_alloc(ctx, sizeof(BuildJob) * jobs.size(), s, &b->jobs_dev))) return fail(st);
        if ((st = upload(ctx, b->jobs_dev, jobs.data(), sizeof(BuildJob) * jobs.size(), s)))
            return fail(st);
        b->n_jobs = (int)jobs.size();
        b->build_blocks = blocks;
    }
    b->grid = P.grid;
    b->threads = P.threads;
    b->R = P.R;
    b->smem = P.smem;
    b->total_pairs = P.total_pairs;
    b->total_fold = P.total_fold;
    b->total_anchor_segs = P.total_anchor_segs;
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(FEW_ERR_CUDA);
    if (!(flags & FEW_BATCH_NO_GRAPH)) {
        cudaStream_t cap = nullptr;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return fail(FEW_ERR_CUDA);
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const PlanHdr *hd = static_cast<const PlanHdr *>(b->blob_dev);
            if (b->n_jobs)
                launch_build(static_cast<const BuildJob *>(b->jobs_dev), b->n_jobs, b->build_blocks,
                             b->max_knots, ctx->d_err, cap);
            // the same fork and join as launch_kernels, recorded into the graph
            const bool fork = b->total_anchor_segs > 0;
            auto &L = ctx->lanes[ctx->lane_next++ % 4];
            if (fork) {
                cudaEventRecord(L.fork, cap);
                cudaStreamWaitEvent(L.s, L.fork, 0);
                launch_anchor(hd, b->total_anchor_segs, L.s);
                cudaEventRecord(L.join, L.s);
            }
            launch_ylm(hd, b->total_pairs, b->fp64, cap);
            launch_fold(hd, b->total_fold, b->fp64, cap);
            if (fork) cudaStreamWaitEvent(cap, L.join, 0);
            launch_sum(hd, b->grid, b->threads, b->R, b->smem, b->variant, cap);
            e = cudaStreamEndCapture(cap, &b->graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return fail(FEW_ERR_CUDA);
    }
    ctx->batches.insert(b);
    *out = b;
    return FEW_OK;
}

few_status few_batch_run(few_ctx *ctx, few_batch *b, void *stream)
{
    NvtxRange nvtx_range("few_batch_run");
    if (!ctx || !b || b->ctx != ctx) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (b->exec) {
        FEW_CUDA_TRY(cudaGraphLaunch(b->exec, s));
        return FEW_OK;
    }
    const PlanHdr *hd = static_cast<const PlanHdr *>(b->blob_dev);
    if (b->n_jobs) {
        tmark(ctx, 0, false, s);
        FEW_CUDA_TRY(launch_build(static_cast<const BuildJob *>(b->jobs_dev), b->n_jobs,
                                  b->build_blocks, b->max_knots, ctx->d_err, s));
        tmark(ctx, 0, true, s);
    }
    return launch_kernels(ctx, hd, b->total_pairs, b->total_fold, b->total_anchor_segs, b->grid,
                          b->threads, b->R, b->smem, b->variant, s);
}

few_status few_batch_release(few_ctx *ctx, few_batch *b)
{
    if (!ctx || !b || b->ctx != ctx) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    // The caller guarantees the batch's work has completed (an event, a stream sync); no device
    // synchronisation here, so other work in flight keeps running.
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    dev_free(ctx, b->jobs_dev, ctx->internal);
    dev_free(ctx, b->scratch_dev, ctx->internal);
    dev_free(ctx, b->blob_dev, ctx->internal);
    cudaStreamSynchronize(ctx->internal);
    (void)cudaGetLastError();
    ctx->batches.erase(b);
    delete b;
    return FEW_OK;
}

few_status few_sync_status(few_ctx *ctx)
{
    if (!ctx) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        (void)cudaGetLastError();
        return FEW_ERR_CUDA;
    }
    unsigned bits = 0;
    if (cudaMemcpy(&bits, ctx->d_err, sizeof(bits), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FEW_ERR_CUDA;
    if (bits && cudaMemset(ctx->d_err, 0, sizeof(unsigned)) != cudaSuccess) return FEW_ERR_CUDA;
    if (bits & ERRBIT_TIMEOUT) return FEW_ERR_TIMEOUT;
    if (bits & ERRBIT_NONFINITE) return FEW_ERR_INVALID_ARG;
    if (bits & ERRBIT_INTERNAL) return FEW_ERR_CUDA;
    return FEW_OK;
}

few_status few_selftest_wait_expiry(few_ctx *ctx, unsigned limit_us, void *stream)
{
    if (!ctx || limit_us < 1 || limit_us > 2000000u) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    FEW_CUDA_TRY(launch_wait_selftest(ctx->d_err, limit_us, static_cast<cudaStream_t>(stream)));
    return FEW_OK;
}

few_status few_ctx_set_timing(few_ctx *ctx, int enable)
{
    if (!ctx) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->timing = enable != 0;
    for (bool &r : ctx->trec) r = false;
    return FEW_OK;
}

few_status few_last_timing(few_ctx *ctx, float *ms)
{
    if (!ctx || !ms) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DeviceScope dev_scope(ctx->device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    for (int i = 0; i < 4; ++i) {
        ms[i] = -1.0f;
        if (!ctx->trec[i]) continue;
        FEW_CUDA_TRY(cudaEventSynchronize(ctx->tev[2 * i + 1]));
        FEW_CUDA_TRY(cudaEventElapsedTime(&ms[i], ctx->tev[2 * i], ctx->tev[2 * i + 1]));
    }
    return FEW_OK;
}

few_status few_set_tiles(few_ctx *ctx, int prec, int R, int threads, int stage_slots)
{
    if (!ctx) return FEW_ERR_INVALID_ARG;
    if (threads != 128 && threads != 256) return FEW_ERR_INVALID_ARG;
    if (prec == FEW_FP64) {
        if (R != 1 && R != 2) return FEW_ERR_INVALID_ARG;
    } else if (prec == FEW_MIXED) {
        if (R != 2 && R != 4 && R != 8) return FEW_ERR_INVALID_ARG;
    } else {
        return FEW_ERR_INVALID_ARG;
    }
    if (stage_slots < kMinStageSlots || stage_slots > kMaxStageSlots || stage_slots % 16)
        return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->tile_R[prec] = R;
    ctx->tile_T[prec] = threads;
    ctx->tile_S[prec] = stage_slots;
    return FEW_OK;
}

few_status few_get_tiles(few_ctx *ctx, int prec, int *R, int *threads, int *stage_slots)
{
    if (!ctx || (prec != FEW_FP64 && prec != FEW_MIXED)) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (R) *R = ctx->tile_R[prec];
    if (threads) *threads = ctx->tile_T[prec];
    if (stage_slots) *stage_slots = ctx->tile_S[prec];
    return FEW_OK;
}

few_status few_plan_segments(const double *t_knots, int K, double t0, double dt, int64_t n_samples,
                             int64_t *seg_start)
{
    if (!seg_start) return FEW_ERR_INVALID_ARG;
    return segments(t_knots, K, t0, dt, n_samples, seg_start);
}

few_status few_mode_slots(const int *l, const int *m, const int *n, int N, int *n_slots, int *n_rows)
{
    SlotPlan P;
    few_status st = plan_slots(l, m, n, N, P);
    if (st) return st;
    if (n_slots) *n_slots = P.n_slots;
    if (n_rows) *n_rows = (int)P.rows.size();
    return FEW_OK;
}

few_status few_plan_cta_slices(int n_waves, const int64_t *seg_start, const int *K,
                               const int *n_slots, int grid, int pass, int *out_wave,
                               int *out_sample)
{
    if (!seg_start || !K || !n_slots || !out_wave || !out_sample || n_waves < 1 || grid < 1 ||
        pass < 1)
        return FEW_ERR_INVALID_ARG;
    std::vector<const int64_t *> segs(n_waves);
    size_t off = 0;
    for (int q = 0; q < n_waves; ++q) {
        if (K[q] < 2 || n_slots[q] < 1) return FEW_ERR_INVALID_ARG;
        segs[q] = seg_start + off;
        for (int k = 0; k + 1 < K[q]; ++k)
            if (segs[q][k + 1] < segs[q][k] || segs[q][k] < 0) return FEW_ERR_INVALID_ARG;
        if (segs[q][K[q] - 1] > 2147483647LL) return FEW_ERR_INVALID_ARG;
        off += (size_t)K[q];
    }
    std::vector<CtaStart> cta((size_t)grid + 1);
    partition_ctas(n_waves, segs.data(), K, n_slots, grid, pass, cta.data());
    for (int g = 0; g <= grid; ++g) {
        out_wave[g] = cta[g].wave;
        out_sample[g] = cta[g].sample;
    }
    return FEW_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------ read-only views
// Used by the allocation-free entry point (noalloc.cu), which plans a request itself.

namespace fewsum {

bool ctx_traj_view(few_ctx *ctx, const few_traj *tr, CtxTrajView *v)
{
    if (!ctx || !tr || !v || tr->ctx != ctx) return false;
    v->device = ctx->device;
    v->sm_count = ctx->sm_count;
    v->d_err = ctx->d_err;
    v->tile_R[0] = ctx->tile_R[0];
    v->tile_R[1] = ctx->tile_R[1];
    v->tile_T[0] = ctx->tile_T[0];
    v->tile_T[1] = ctx->tile_T[1];
    v->tile_S[0] = ctx->tile_S[0];
    v->tile_S[1] = ctx->tile_S[1];
    v->has_data = tr->has_data;
    v->K = tr->K;
    v->n_slots = tr->plan.n_slots;
    v->n_pairs = (int)tr->plan.pair_lm.size();
    v->t_host = tr->t_host.data();
    v->dev = tr->dev;
    return true;
}

std::recursive_mutex &ctx_mutex(few_ctx *ctx) { return ctx->mu; }

few_status check_request(const few_request &r, bool need_device_out)
{
    return validate_request(r, need_device_out);
}

}  // namespace fewsum
