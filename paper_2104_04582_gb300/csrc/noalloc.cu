// noalloc.cu -- few_waveform_noalloc: one waveform without any memory allocation.
//
// Why it exists: some callers may not allocate device memory on the call path at all -- for
// example a sampler or a real-time pipeline that reserves every byte at start-up and must not
// touch the allocator (or its synchronisation) afterwards, or host code running under a
// memory policy where cudaMalloc is forbidden after initialisation.  few_waveform takes its
// scratch (the plan, the harmonic table and the folded coefficients) from the context's pool on
// every call; this entry point instead places all of that in one fixed device array that is
// part of the library image, so a call performs no allocation of any kind.
//
// The array (kScratchBytes, 16 MiB) is reserved on every GPU that loads the library and stays
// there until the process exits.  Its address is looked up once per device with
// cudaGetSymbolAddress during the first call made with that device current; that first call
// should therefore come before any stream capture.  All calls share the array: nothing in it
// has to start at zero (every call rewrites the whole region it uses before reading it), but
// two calls whose work overlaps on the GPU (different streams, no ordering) race on it.
#include <cmath>
#include <cstring>
#include <mutex>

#include "fewsum_internal.h"

namespace fewsum {

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // FEW_NOALLOC_SCRATCH_BYTES
constexpr int kMaxDevices = 64;
constexpr int kMaxKnots = 4096;
constexpr int kMaxGrid = 4096;
constexpr int kChunk = 3072;  // plan bytes carried by one copy launch (kernel parameters)
constexpr size_t kBlobMax = 64 * 1024;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host-side table of the array's device address, per device.
std::mutex g_setup_mu;
void *g_scratch_dev[kMaxDevices] = {};

// Host image of one plan, rebuilt under a lock on every call (no heap use).
std::mutex g_blob_mu;
alignas(256) unsigned char g_blob[kBlobMax];

struct ChunkParams {
    unsigned char bytes[kChunk];
};

// Copies one chunk of the plan, passed by value as kernel parameters, into the array.
__global__ void k_put_chunk(unsigned char *dst, ChunkParams p, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = p.bytes[i];
}

inline size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

few_status scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) return FEW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return FEW_ERR_CUDA;
        }
        g_scratch_dev[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_dev[device]);
    return FEW_OK;
}

}  // namespace

}  // namespace fewsum

using namespace fewsum;

extern "C" few_status few_waveform_noalloc(few_ctx *ctx, const few_request *req, void *stream)
{
    if (!ctx || !req || !req->traj || !req->out) return FEW_ERR_INVALID_ARG;
    const few_request &r = *req;
    std::lock_guard<std::recursive_mutex> lk(ctx_mutex(ctx));
    CtxTrajView v;
    if (!ctx_traj_view(ctx, r.traj, &v)) return FEW_ERR_INVALID_ARG;
    few_status st = check_request(r, true);  // as few_waveform; device output only
    if (st) return st;
    const int K = v.K, S = K - 1;
    const bool fp64 = r.prec == FEW_FP64;
    if (K > kMaxKnots) return FEW_ERR_LIMIT;
    if (r.n_samples == 0) return FEW_OK;
    DeviceScope dev_scope(v.device);
    if (!dev_scope.ok) return FEW_ERR_CUDA;
    unsigned char *base = nullptr;
    if ((st = scratch_address(v.device, &base))) return st;

    // tile shape and grid as in few_waveform
    const int pi = fp64 ? 0 : 1;
    const int R = v.tile_R[pi], T = v.tile_T[pi];
    const int variant = fp64 ? kVariantFp64 : kVariantScalar;
    const size_t slot_bytes = (size_t)sum_slot_bytes(variant);
    const int stage_slots = v.tile_S[pi] < v.n_slots ? v.tile_S[pi] : v.n_slots;
    const int buf_bytes = (int)up((size_t)stage_slots * slot_bytes, 128);
    const int smem = kDefaultRing * buf_bytes;
    const int occ = sum_occupancy(variant, R, T, smem);
    if (occ <= 0) return FEW_ERR_LIMIT;
    const int grid = v.sm_count * occ;
    if (grid > kMaxGrid) return FEW_ERR_LIMIT;

    // layout inside the fixed array: [plan | folded coefficients | harmonic table | anchors]
    const size_t off_waves = up(sizeof(PlanHdr), 64);
    const size_t off_cta = up(off_waves + sizeof(WaveDev), 64);
    const size_t off_seg = up(off_cta + sizeof(CtaStart) * (grid + 1), 64);
    const size_t off_anc = up(off_seg + sizeof(int) * K, 64);
    const size_t blob_bytes = up(off_anc + (fp64 ? 0 : sizeof(int) * K), 256);
    if (blob_bytes > kBlobMax) return FEW_ERR_LIMIT;

    std::lock_guard<std::mutex> blk(g_blob_mu);
    std::memset(g_blob, 0, blob_bytes);
    PlanHdr *hdr = reinterpret_cast<PlanHdr *>(g_blob);
    WaveDev *W = reinterpret_cast<WaveDev *>(g_blob + off_waves);
    CtaStart *cta = reinterpret_cast<CtaStart *>(g_blob + off_cta);
    int *seg = reinterpret_cast<int *>(g_blob + off_seg);
    int *anc = reinterpret_cast<int *>(g_blob + off_anc);

    // segment sample ranges: seg[k] = clamp(ceil((t_k - t0)/dt), 0, n)
    const int64_t ns = r.n_samples;
    seg[0] = 0;
    for (int k = 1; k < K - 1; ++k) {
        const double x = std::ceil((v.t_host[k] - r.t0) / r.dt);
        int64_t val = x <= 0.0 ? 0 : (x >= (double)ns ? ns : (int64_t)x);
        if (val < seg[k - 1]) val = seg[k - 1];
        seg[k] = (int)val;
    }
    seg[K - 1] = (int)ns;
    // mixed path: first phase anchor of each segment, then the total
    int n_anchors = 0;
    if (!fp64) {
        for (int k = 0; k + 1 < K; ++k) {
            anc[k] = n_anchors;
            n_anchors += anchors_in_segment(seg[k], seg[k + 1]);
        }
        anc[K - 1] = n_anchors;
    }
    const size_t fcoef_bytes = up((size_t)S * v.n_slots * slot_bytes, 256);
    const size_t ylm_bytes = up((size_t)v.n_pairs * 2 * sizeof(double2), 256);
    const size_t anc_bytes = up(sizeof(Anchor) * (size_t)n_anchors, 256);
    if (blob_bytes + fcoef_bytes + ylm_bytes + anc_bytes > kScratchBytes) return FEW_ERR_LIMIT;
    unsigned char *d_fcoef = base + blob_bytes;
    unsigned char *d_ylm = d_fcoef + fcoef_bytes;
    unsigned char *d_anc = d_ylm + ylm_bytes;

    W->tr = v.dev;
    W->theta = r.theta;
    W->phi = r.phi;
    W->scale = r.scale;
    W->dphi_phi = r.dphi_phi0;
    W->dphi_r = r.dphi_r0;
    W->t0 = r.t0;
    W->dt = r.dt;
    W->n_samples = (int)ns;
    W->out_c64 = r.out_c64 ? 1 : 0;
    W->out = r.out;
    W->frame = r.frame;
    W->theta_K = r.theta_K;
    W->phi_K = r.phi_K;
    W->fcoef = d_fcoef;
    W->ylm = reinterpret_cast<double2 *>(d_ylm);
    W->seg_start = reinterpret_cast<const int *>(base + off_seg);
    W->pair_begin = 0;
    W->fold_begin = 0;
    W->fold_blocks_per_seg = (v.n_slots + kFoldThreads - 1) / kFoldThreads;
    if (!fp64) {
        W->anchors = reinterpret_cast<Anchor *>(d_anc);
        W->anchor_off = reinterpret_cast<const int *>(base + off_anc);
        W->anchor_seg_begin = 0;
    }

    // equal slices of the samples (one waveform: equal cost per sample)
    for (int g = 0; g < grid; ++g) {
        const long double x = (long double)ns * g / grid;
        cta[g] = CtaStart{0, (int)std::ceil(x)};
    }
    cta[grid] = CtaStart{1, 0};

    hdr->n_waves = 1;
    hdr->total_pairs = v.n_pairs;
    hdr->total_fold_blocks = S * W->fold_blocks_per_seg;
    hdr->total_anchor_segs = fp64 ? 0 : S;
    hdr->grid_sum = grid;
    hdr->buf_bytes = buf_bytes;
    hdr->stage_slots = stage_slots;
    hdr->ring = kDefaultRing;
    hdr->variant = variant;
    hdr->waves = reinterpret_cast<const WaveDev *>(base + off_waves);
    hdr->cta = reinterpret_cast<const CtaStart *>(base + off_cta);
    hdr->err = v.d_err;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (size_t off = 0; off < blob_bytes; off += kChunk) {
        const int n = (int)((blob_bytes - off) < (size_t)kChunk ? (blob_bytes - off) : kChunk);
        ChunkParams p;
        std::memcpy(p.bytes, g_blob + off, (size_t)n);
        k_put_chunk<<<1, 256, 0, s>>>(base + off, p, n);
    }
    if (cudaGetLastError() != cudaSuccess) return FEW_ERR_CUDA;
    const PlanHdr *hd = reinterpret_cast<const PlanHdr *>(base);
    if (launch_ylm(hd, v.n_pairs, fp64, s) != cudaSuccess ||
        launch_fold(hd, hdr->total_fold_blocks, fp64, s) != cudaSuccess ||
        launch_anchor(hd, fp64 ? 0 : S, s) != cudaSuccess ||
        launch_sum(hd, grid, T, R, smem, variant, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return FEW_ERR_CUDA;
    }
    return FEW_OK;
}
