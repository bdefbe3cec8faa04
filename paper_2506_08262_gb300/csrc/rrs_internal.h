// Internal structures shared by the host runtime (rrs_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rrs.h"

namespace rrs {

// A resident dataset, as the kernels see it.
struct DsDev {
    const float* X32;      // n x ldx FP32 rows, zero padded
    // Xt: the FP32 rows again, for the selection kernels' projection pass (d <= 16), or nullptr.  Rows come in
    // tiles of 32 (the last one zero padded); within a tile, 16-byte chunk c of its 32 rows is contiguous:
    // float4 index ((i / 32) * (ldx / 4) + c) * 32 + i % 32.  A warp reading chunk c of 32 consecutive rows
    // then reads 512 contiguous bytes (4 cache lines) where padded rows spread it over all 12 lines of d = 10.
    const float* Xt;
    const double* X64;     // n x d FP64 rows, or nullptr if the data came in FP32
    const float* xnorm;    // n Euclidean row norms, rounded up
    const uint16_t* Xbf;   // n x (2*kp) BF16 planes [x_hi | x_lo] for the tensor-core path, or nullptr
    const float* center;   // d: mean of the rows
    const float* cov;      // d x d covariance of the rows (d <= RRS_COV_MAX_D), else nullptr
    int64_t n;
    int32_t d;
    int32_t ldx;           // padded FP32 row stride (floats)
    int32_t kp;            // padded K of one BF16 plane (multiple of 64), 0 if no planes
    float rc;              // max_i |x_i - center| (rounded up): every |u'(x_i - center)| <= rc for |u| <= 1
};

constexpr int RRS_COV_MAX_D = 128;

// One query of a launch (any request, any dataset).
struct SlotDev {
    int32_t ds;            // index into the DsDev array
    int32_t kind;
    int32_t m;             // directions per round
    int32_t r;             // rounds
    float alpha;
    int32_t d;
    int32_t ldx;
    int32_t zdtype;        // 0 = FP32, 1 = FP64
    uint64_t seed;
    int64_t qctr;          // query counter index in the direction stream
    int64_t uoff;          // offset of this slot's m x ldx directions in U (floats)
    int64_t roff;          // offset of this slot's m results / y_z values
    int64_t zoff32;        // offset of the FP32 query row (ldx floats) and of the poles
    int64_t zoff64;        // offset of the FP64 query row (d doubles)
    const void* zsrc;      // caller's query row (device)
    double* depth_out;     // this query's output cells (device), may be null
    int64_t* count_out;
    int32_t* best_out;
    int32_t* choice_out;   // r cells
    // running state (Alg. 1 step 5)
    double dmin;
    int64_t cmin;
    int32_t best;
    float znorm;
    int32_t round;         // next round (0-based) when launched in per-slot round mode
    int32_t pad2;
};

// A block of directions of one slot handled by one CTA.
struct TaskDev {
    int32_t slot;
    int32_t j0;
    int32_t nj;
    int32_t ds;            // selection tasks: the slot's dataset row (read beside the slot, not after it); else 0
};

// Per (slot, direction) result of one round.
struct ResDev {
    double depth;
    int64_t count;         // halfspace: min(#<=, #>=); else -1
};

// Device-side error bits (ORed into one word).
enum : int {
    ERR_SELECT_ITER = 1,    // bucket selection did not converge
    ERR_SELECT_CAP = 2,
    ERR_EXPANSION = 4,      // exact-sign expansion overflow
    ERR_TIMEOUT = 8,
    ERR_TC_SETUP = 16,
};

// Near-tie band factors: a point is re-checked exactly when
// |t| <= gamma * (|x| + |z|), t the fast projection difference.
// FP32 path: |fl32 dot - exact| <= gamma_d sum|u x| (gamma_d ~ d 2^-24), plus one rounding of x to FP32
// (FP64 inputs), of y_z to FP32 and of the final difference; twice that sum for slack.
__host__ __device__ inline float band_gamma_fp32(int d) { return (float)((double)(d + 4) * 0x1p-23); }
float band_gamma_tc(int kp);
// cuTensorMapEncodeTiled, looked up once through the runtime (NULL when unavailable)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn();
__host__ __device__ float band_coef_ff(int d);   // bound coefficient of the compensated FP32 re-check (tensor-core path)

// Set the text that rrs_last_error() returns on this thread (rrs_api.cu).
void set_last_error(const char* msg);

// launchers (rrs_kernels.cu)
cudaError_t launch_prep(const SlotDev* slots, int nslots, const DsDev* ds, float* z32, double* z64,
                        float* poles, cudaStream_t st);
// max_ldx: the largest row stride among the tasks' queries (sizes the shared-memory staging)
cudaError_t launch_gen(const TaskDev* tasks, int ntasks, const SlotDev* slots, const float* poles_cur,
                       const double* z64, float* U, double* yz, int round0, int max_ldx, cudaStream_t st);
cudaError_t launch_hd_simt(const TaskDev* tasks, int ntasks, int max_ldx, const SlotDev* slots, const DsDev* ds,
                           const float* U, const double* yz, const double* z64, ResDev* res, int64_t* band_out,
                           int* err, cudaStream_t st);
// group: directions per CTA (1, 2 or 4, from pdap_shape); variant: pdap_shape's kernel variant (the key
// arithmetic class pdap_dp4_class(d), plus PDAP_STREAM), shared by every task
// yz: the FP64 y_z = u'z of every direction (the direction generator's output), used for the depth.
// Launches the selection kernel, which writes the points holding the order statistics into the result cells,
// then k_pdap_finish, which forms the depths from FP64 projections of those points: PDAP_LAUNCH_KERNELS kernels.
constexpr int PDAP_LAUNCH_KERNELS = 2;
cudaError_t launch_pdap(const TaskDev* tasks, int ntasks, size_t smem, int group, int variant, const SlotDev* slots,
                        const DsDev* ds, const float* U, const double* yz, ResDev* res, int* err, cudaStream_t st,
                        const float* kin = nullptr);
// Keys of ntasks selection tasks (all of one dataset) into keys (pdap_keys_bytes), for
// launch_pdap(..., kin = keys) on the same task range, with the selection kernel's own key arithmetic:
// a tiled FP32 GEMM for d > 16 (where forming the keys inside the selection kernel re-reads X for every
// G directions), two half chains per key for d <= 16 (used when the keys do not fit shared memory)
size_t pdap_keys_bytes(int n, int group, int ntasks);
cudaError_t launch_pdap_keys(const TaskDev* tasks, int ntasks, int group, const SlotDev* slots, const DsDev* ds,
                             const DsDev& ds_host, const float* U, float* keys, cudaStream_t st);
int pdap_dp4_class(int d);
cudaError_t launch_argmin(SlotDev* slots, const int32_t* slot_list, int nlist, const float* U,
                          const ResDev* res, const float* poles_cur, float* poles_next, int round0,
                          int last_round, cudaStream_t st);
cudaError_t launch_yz_only(const TaskDev* tasks, int ntasks, const SlotDev* slots, const double* z64,
                           const float* U, double* yz, cudaStream_t st);
cudaError_t launch_scatter_dirs(const SlotDev* slots, int nslots, int m, int d, const float* Uin, float* U,
                                cudaStream_t st);
// Per-slot round mode (serving): each slot runs its own next round S.round; poles0 holds the
// pole of slots at even rounds, poles1 of odd ones; argmin advances S.round.
cudaError_t launch_gen_slotround(const TaskDev* tasks, int ntasks, const SlotDev* slots, const float* poles0,
                                 const float* poles1, const double* z64, float* U, double* yz, int max_ldx,
                                 cudaStream_t st);
cudaError_t launch_argmin_slotround(SlotDev* slots, const int32_t* slot_list, int nlist, const float* U,
                                   const ResDev* res, float* poles0, float* poles1, cudaStream_t st);
cudaError_t launch_debug_dirs(uint64_t seed, int q, int round0, int m, int d, float alpha, const float* pole,
                              float* U, cudaStream_t st);
cudaError_t launch_convert_dataset(const void* X, int dtype, int64_t n, int d, int ldx, float* X32,
                                   double* X64, float* xnorm, int* bad, cudaStream_t st);
// DsDev::Xt from the padded rows X32 (Xt holds tile_rows_floats(n, ldx) floats)
size_t tile_rows_floats(int64_t n, int ldx);
cudaError_t launch_tile_rows(const float* X32, int64_t n, int ldx, float* Xt, cudaStream_t st);
// mean, covariance (d <= RRS_COV_MAX_D) and radius about the mean of the FP32 rows; rc_out is a device float
cudaError_t launch_moments(const float* X32, int64_t n, int d, int ldx, float* center, float* cov, float* rc_out,
                           cudaStream_t st);
cudaError_t launch_check_finite(const void* Z, int dtype, int64_t count, int* bad, cudaStream_t st);
size_t pdap_smem_bytes(int n, int group, int ldx, bool stream = false);
size_t pdap_smem_limit();
// preferred resident G; 0: keys outside shared memory (when allow_stream, or when none fits)
int pdap_max_group(int n, int ldx, int m, int d, bool keys_in = false, bool allow_stream = false);

// Selection-kernel variant bit: the keys are not held in shared memory (n beyond what shared memory holds
// for one direction); every pass reads them from k_keys output in global memory when given (kin), else
// recomputes them from X.  Such launches take PDAP_STREAM_GROUP directions per CTA.
constexpr int PDAP_STREAM = 0x100;
// Largest n the selection kernels take: point indices and the padded key count (n rounded up to 4) are int.
constexpr int64_t PDAP_MAX_N = 0x7FFFFFC0;
constexpr int PDAP_STREAM_GROUP = 2;
// Selection-kernel variant bit: one warp per direction, up to PDAPW_DIRS directions per CTA, keys re-formed
// from X at every pass (d <= 16, n <= PDAPW_MAX_N: 16-bit bucket counters); the low byte holds d.  Asking
// pdap_shape for group PDAP_WARP_GROUP selects it where it applies.
constexpr int PDAP_WARP = 0x200;
constexpr int PDAPW_DIRS = 12;
constexpr int64_t PDAPW_MAX_N = 12288;
constexpr int PDAP_WARP_GROUP = RRS_SELECT_WARP;
// pdap_shape group asking for the keys outside shared memory (formed once per round, read at every pass)
constexpr int PDAP_STREAM_CHOICE = RRS_SELECT_STREAM;
size_t pdapw_smem_bytes(int d);
bool pdapw_eligible(int64_t n, int d);
struct PdapShape {
    int group;        // directions per CTA
    int variant;      // pdap_dp4_class(d), plus PDAP_STREAM; or PDAP_WARP | d
    size_t smem;      // dynamic shared memory per CTA
    bool keys_gemm;   // keys formed first by launch_pdap_keys
};
// Launch shape for a dataset (n rows, d dims, row stride ldx) and m directions per query; group > 0 asks for
// that many resident directions per CTA (taken when it fits), 0 picks by the shared-memory heuristic.
PdapShape pdap_shape(int n, int ldx, int m, int d, int group = 0);

// tensor-core path (hd_tc.cu)
cudaError_t launch_build_bf16_planes(const float* X32, int64_t n, int d, int ldx, int kp, uint16_t* Xbf,
                                     cudaStream_t st);
// Points per tile of the tensor-core kernel for planes of K extent kp: want = 128 or 256 where both exist
// (kp = 64), anything else for the default.
int tc_tile_n(int kp, int want = 0);
// The tensor map of a dataset's BF16 planes (kp 64 or 128; planes built) for tiles of bn points, written to *out
// (host memory; the caller copies it into the device array passed as maps).
cudaError_t encode_tc_map(const DsDev& ds_host, int bn, CUtensorMap* out);
// tasks of up to 128 (query, direction) rows each, of any datasets whose planes have K extent kp and whose maps
// were encoded for tiles of bn points; maps[ds] is the tensor map of dataset row ds of ds_dev (device memory,
// 64-byte aligned)
cudaError_t launch_hd_tc(const TaskDev* tasks, int ntasks, int kp, int bn, const SlotDev* slots,
                         const DsDev* ds_dev, const CUtensorMap* maps, const float* U, const double* yz,
                         const double* z64, ResDev* res, int64_t* band_out, int* err, cudaStream_t st);
bool hd_tc_supported(int d);
cudaError_t launch_wait_probe(int* err, long long limit_cycles, cudaStream_t st);

}  // namespace rrs
