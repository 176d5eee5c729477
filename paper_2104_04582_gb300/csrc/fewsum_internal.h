// fewsum_internal.h -- device-side descriptors shared by the host API (api.cpp) and the
// kernels (spline.cu, fold.cu, sum.cu).  Plain structs: the host fills them, uploads them in
// one plan blob per call or batch, and the kernels read them.
#pragma once

#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "fewsum.h"

namespace fewsum {

// Device error latch bits (few_ctx::d_err); decoded by few_sync_status.
enum : unsigned {
    ERRBIT_NONFINITE = 1u,  // non-finite value in device-resident inputs
    ERRBIT_TIMEOUT = 2u,    // a bounded mbarrier wait expired
    ERRBIT_INTERNAL = 4u    // a decoded index fell outside its table (should not happen)
};

constexpr int kMaxL = 32;
constexpr int kMaxAbsN = 1024;
// Summation kernel: up to kSumMaxThreads threads per CTA; the per-segment slot table streams
// through a ring of shared-memory stages of stage_slots slots each.
constexpr int kSumMaxThreads = 256;
constexpr int kMaxRing = 4;
constexpr int kDefaultRing = 3;
constexpr int kMinStageSlots = 16, kMaxStageSlots = 4096;

// Summation kernel variants (and the folded-coefficient layout each reads).
enum : int {
    kVariantFp64 = 0,   // FP64 throughout; slot = 8 doubles
    kVariantScalar = 1  // mixed: FP64 phases at anchors, FP32 everything else; slot = 8 floats
};

// Phase anchors of the mixed path: the FP64 phase splines are evaluated and reduced modulo one
// turn at every kAnchorGroup-th sample (absolute sample index a = kAnchorGroup * q), together
// with the exact Taylor coefficients of the phase cubic about that sample in sample units; the
// summation kernel adds the increment to the following samples of the group in FP32.
constexpr int kAnchorGroup = 16;
constexpr int kAnchorThreads = 128, kAnchorBlocksPerSeg = 4;  // anchor kernel grid per segment
struct Anchor {
    float4 phi;  // (f0, d1, d2, d3): reduced phase (turns) and increment coefficients (turns / sample^k)
    float4 r;
    float4 g;    // phase of the final factor z_phi^{m_last} z_r^{lo_last}, same form
};
constexpr int kFoldThreads = 128;
constexpr int kYlmThreads = 16;  // few pairs per block: spreads the FP64 work over SMs
constexpr int kBuildThreads = 64;
constexpr int kBuildParts = 8;  // blocks of a spline's partitioned solve = lanes per spline
constexpr int kBuildSplines = kBuildThreads / kBuildParts;

// Trajectory-resident data (one per few_traj).
struct TrajDev {
    int K, N, J, S;        // knots, modes, splines (2 + 2N), segments (K - 1)
    int n_pairs;           // distinct (l, m) pairs
    int n_slots;           // harmonic slots per segment
    int n_rows;            // rows of the slot table: signed m from max m down to m_last
    int m_last, lo_last;   // signed m and lowest n of the last row
    const double *t;       // [K] knot times
    const double *inv_h;   // [S] 1/(t_{k+1}-t_k)
    const double *h;       // [S] t_{k+1}-t_k
    // the partitioned factorisation of the reduced not-a-knot system (k_factor); p_k = pivot
    const double *fac_ra;  // [K] right-hand side f_k = ra_k (y_k - y_{k-1}) + rb_k (y_{k+1} - y_k):
    const double *fac_rb;  //   block rows scaled by 1/p_k, separator rows plain; rows 0 and K-1
                           //   hold the end slopes' coefficients (see k_factor)
    const double *fac_lo;  // [K] block rows: sub-diagonal / p_k (0 on a block's first row);
                           //   rows 0 and K-1: the end slopes' coupling to s_1 / s_{K-2}
    const double *fac_up;  // [K] block rows: super-diagonal / p_k
    const double *fac_ip;  // [K] inverse pivots (block rows; separator system at separator rows)
    const double *fac_v;   // [K] block responses v to the left separator (separator multipliers)
    const double *fac_x;   // [K] block responses w to the right separator (separator couplings)
    const double *fac_sinv;  // [(kBuildParts-1)^2] inverse of the separator system, row-major
    const int *parts;      // [kBuildParts + 2]: block count P, block starts, then K - 1
    double *slopes;        // [K][J] spline build scratch (parked elimination values)
    double *coef;          // [S][J][4] Hermite data of every segment: (y_k, y_{k+1}, s_k,
                           //   s_{k+1}), values and knot slopes (see hermite_to_power);
                           //   columns 0,1 = Phi_phi, Phi_r (rad),
                           //   column 2+2i / 3+2i = Re / Im A_i
    const int2 *pair_lm;   // [n_pairs] (l, m)
    const int *mode_pair;  // [N] pair index of each mode
    const int *slot_ptr;   // [n_slots + 1] CSR into contrib
    const int2 *contrib;   // [n_contrib] (mode * 2 + kind, 2 * pair + kind); kind 0: A Y+,
                           //   1: conj(A) Y-
    const int2 *rows;      // [n_rows] (slots of the row, lowest n of the previous row minus
                           //   this row's lowest n); a row's slots run from its highest n down
};

// Power coefficients of a segment's cubic in the local variable u = (t - t_k)/h_k, u in [0, 1],
// from its Hermite data (values y0 = y_k, y1 = y_{k+1}, slopes s0, s1, width h = h_k):
//     p(u) = y0 + a u + (3 D - 2 a - b) u^2 + (a + b - 2 D) u^3,  a = h s0, b = h s1, D = y1 - y0.
template <typename T>
__host__ __device__ __forceinline__ void hermite_to_power(T y0, T y1, T s0, T s1, T h, T (&c)[4])
{
    const T D = y1 - y0, a = h * s0, b = h * s1;
    c[0] = y0;
    c[1] = a;
    c[2] = fma((T)-2, a, fma((T)3, D, -b));
    c[3] = fma((T)-2, D, a + b);
}

// One spline-build job: a trajectory and the knot data to fit.
struct BuildJob {
    TrajDev tr;
    const double *phi_phi;  // [K] rad
    const double *phi_r;    // [K] rad
    const double *amp_re;   // [K][N]
    const double *amp_im;   // [K][N]
    int block_begin;        // first block of this job in the flattened build grid
    int pad;
};

// One waveform of a plan (a request).
struct WaveDev {
    TrajDev tr;
    double theta, phi, scale;
    double dphi_phi, dphi_r;    // phase offsets (rad)
    double t0, dt;
    int n_samples;
    int out_c64;
    void *out;
    void *fcoef;          // [S][n_slots][8] folded coefficients (float or double)
    Anchor *anchors;      // mixed plans: [n_anchors] phase anchors (segment by segment)
    const int *anchor_off;  // mixed plans: [K] first anchor of each segment, then the total
    int anchor_seg_begin; // first global segment index of this wave (anchor kernel grid)
    double2 *ylm;         // [n_pairs][2]: Y+ = -2Y_{l,m}, Y- = (-1)^l -2Y_{l,-m} (0 if m = 0)
    const int *seg_start; // [K] sample range of each segment
    int pair_begin;       // first global pair index of this wave (ylm kernel)
    int fold_begin;       // first fold block of this wave
    int fold_blocks_per_seg;
    int frame;            // few_frame: (theta, phi) source-frame angles, or sky position
    double theta_K, phi_K;  // spin direction (frame == FEW_FRAME_SSB)
};

// Start of one CTA's slice of the summation work: (wave, sample).
struct CtaStart {
    int wave;
    int sample;
};

// Header of a plan blob.  The blob is [PlanHdr][WaveDev x n][CtaStart x (grid+1)][ints...].
struct PlanHdr {
    int n_waves;
    int total_pairs;
    int total_fold_blocks;
    int grid_sum;
    int total_anchor_segs;  // segments over all waves of a mixed plan (0 for FP64 plans)
    int buf_bytes;   // bytes of one ring stage (stage_slots x slot bytes, rounded up)
    int stage_slots; // slots per ring stage (the mode tile)
    int ring;        // ring stages
    int variant;     // kVariant* of the summation kernel and the folded layout
    const WaveDev *waves;
    const CtaStart *cta;
    unsigned *err;
};

// Kernel launchers (defined in the .cu files; every launcher returns the launch error).
// Output arrays of k_factor (the trajectory's TrajDev fields of the same names).
struct FactorArrays {
    double *h, *inv_h, *ra, *rb, *lo, *up, *ip, *v, *x, *sinv;
    int *parts;
};
cudaError_t launch_factor(const double *t, int K, const FactorArrays &f, cudaStream_t st);
cudaError_t launch_build(const BuildJob *jobs_dev, int n_jobs, int total_blocks,
                         int max_knots, unsigned *err, cudaStream_t st);
cudaError_t launch_ylm(const PlanHdr *hdr_dev, int total_pairs, bool fp64, cudaStream_t st);
cudaError_t launch_fold(const PlanHdr *hdr_dev, int total_fold_blocks, bool fp64, cudaStream_t st);
cudaError_t launch_anchor(const PlanHdr *hdr_dev, int total_anchor_segs, cudaStream_t st);
// Anchors of one segment's samples [s_begin, s_end): groups floor(s_begin / G) ..
// floor((s_end - 1) / G); none for an empty segment.
inline int anchors_in_segment(int s_begin, int s_end)
{
    return s_end > s_begin ? (s_end - 1) / kAnchorGroup - s_begin / kAnchorGroup + 1 : 0;
}
cudaError_t launch_wait_selftest(unsigned *err, unsigned limit_us, cudaStream_t st);
cudaError_t launch_sum(const PlanHdr *hdr_dev, int grid, int threads, int samples_per_thread,
                       int smem_bytes, int variant, cudaStream_t st);
// Bytes of one folded slot in the layout a variant reads.
int sum_slot_bytes(int variant);
cudaError_t launch_phases(const TrajDev &tr, const int *seg_start, double t0, double dt, int n,
                          double dphi_phi, double dphi_r, double *out, cudaStream_t st);
// Mode Selector: at most kSelectMaxModes modes; which of them stand for an m < 0 partner too
// (m > 0, power doubled) travels as one bit per mode (bit i % 32 of word i / 32) in the launch
// parameters, so a call needs no device allocation or copy.
constexpr int kSelectMaxModes = 4096;
struct ModeDoubling {
    unsigned w[kSelectMaxModes / 32];
};
cudaError_t launch_mode_select(const double *amp_re, const double *amp_im, int K, int N,
                               const ModeDoubling &dbl, double eps, unsigned char *mask,
                               cudaStream_t st);
int mode_select_max_modes();
cudaError_t launch_direct(const double *pphi, const double *pr, const double *are,
                          const double *aim, long long ns, const int *l, const int *m, const int *n,
                          int N, double theta, double phi, double scale, bool fp64, void *out,
                          int out_c64, void *mode_consts, int sm_count, cudaStream_t st);
size_t direct_mode_const_bytes(int N);
// Reduced-basis amplitudes (rb.cu): tile counts of the packed tensor-core operands.
struct RbLayout {
    int n_kb = 0, n_tiles = 0, m_tiles = 0, modes_padded = 0, rows_padded = 0;
    size_t bpack_bytes = 0, apack_bytes = 0;
};
RbLayout rb_layout(int Nb, int N, int M);
cudaError_t launch_rb_basis(const double *bre, const double *bim, int Nb, int N, double2 *gt64,
                            float2 *gt32, int *bexp, unsigned char *bpack, int sm_count, cudaStream_t st);
cudaError_t launch_rb(const double *are, const double *aim, int M, int Nb, int N, const double *nu,
                      bool fp64, const double *bre, const double *bim, const double2 *gt64,
                      const float2 *gt32, const int *bexp, const unsigned char *bpack, double *scale,
                      int *aexp, unsigned char *apack, double *ore, double *oim, unsigned *err,
                      int sm_count, cudaStream_t st, cudaStream_t side, cudaEvent_t fork_ev,
                      cudaEvent_t join_ev);
// Maximum resident CTAs per SM of the summation kernel for a configuration (0 if invalid).
int sum_occupancy(int variant, int samples_per_thread, int threads, int smem_bytes);
// One-time kernel attribute setup (dynamic shared memory opt-in).
cudaError_t sum_configure();

// Makes `device` current for the lifetime of the object and then restores the caller's current
// device, so a library call never leaves a different device current behind.
struct DeviceScope {
    int prev = -1;
    bool ok = false;
    explicit DeviceScope(int device)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            (void)cudaGetLastError();
        }
        ok = cudaSetDevice(device) == cudaSuccess;
        if (!ok) (void)cudaGetLastError();
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
};

// Host validation of one request (few_waveform's checks; need_device_out additionally requires
// out_where == FEW_MEM_DEVICE).
few_status check_request(const few_request &r, bool need_device_out);

// Read-only snapshot of a context and one of its trajectories (filled by api.cpp).
struct CtxTrajView {
    int device, sm_count;
    unsigned *d_err;
    int tile_R[2], tile_T[2], tile_S[2];
    bool has_data;
    int K, n_slots, n_pairs;
    const double *t_host;
    TrajDev dev;
};
bool ctx_traj_view(few_ctx *ctx, const few_traj *tr, CtxTrajView *v);
std::recursive_mutex &ctx_mutex(few_ctx *ctx);

}  // namespace fewsum
