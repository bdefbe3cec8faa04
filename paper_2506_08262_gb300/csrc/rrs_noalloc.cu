// rrs_depth_noalloc: the RRS depth pipeline for callers that must not allocate
// device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// runtime's fixed memory pool, plug-ins whose host forbids allocation after
// start-up, and latency-critical loops that must never hit the allocator.  This
// entry point serves them.  Every piece of working memory the pipeline needs
// (the FP32 copy of X with its row norms, the per-query state, the directions
// of a round and their depths, the launch tables) is carved out of one
// file-scope device array of fixed size, RRS_NOALLOC_SCRATCH_BYTES.  The caller
// passes its inputs and outputs as device pointers; no cudaMalloc, cudaFree or
// other allocating routine is called, on the device or on the host.
//
// The array lives in every device that loads the library until the process
// exits.  In host code its name is only a host-side stand-in, so every call
// asks the runtime for its device address (cudaGetSymbolAddress, with the
// calling device current) and hands that address to the kernels; asking on
// every call keeps the address right even after a cudaDeviceReset.  The first
// call on a device also loads the library's device code there, so that first
// call should come before any stream capture.  All calls share the array and
// it keeps the previous call's contents: the call clears what must start at
// zero, and two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it.  Every call waits for its stream twice
// (to read the input check and the device-side error flags) and returns after
// the stream has finished the work.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>

#include "../../include/rrs.h"
#include "rrs_internal.h"

using namespace rrs;

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[RRS_NOALLOC_SCRATCH_BYTES];

rrs_status noalloc_fail(rrs_status st, const char* fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    set_last_error(msg);   // text returned by rrs_last_error()
    return st;
}

// Device address of the scratch array on the current device.
rrs_status scratch_address(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return noalloc_fail(RRS_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    }
    *out = p;
    return RRS_OK;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

int padded_stride(int d)
{
    int l = (d + 3) & ~3;
    if (((l / 4) & 1) == 0) l += 4;
    return l;
}

struct Layout {
    size_t ds, x32, xnorm, mom, slots, gen, hd, pd, arg, z32, poles, z64, U, yz, res, err, total;
};

Layout layout(int64_t n, int ldx, int d, int64_t nq, int m, int gen_per, int hd_per, int pd_per)
{
    Layout L{};
    size_t o = 0;
    bool over = false;
    // the caller bounds n, nq and nq * m by the scratch size first, so no product below wraps;
    // take() marks the layout as too large once the running total passes the scratch size
    auto take = [&](size_t bytes) {
        const size_t at = o;
        if (bytes > (size_t)RRS_NOALLOC_SCRATCH_BYTES || o + bytes > (size_t)RRS_NOALLOC_SCRATCH_BYTES) over = true;
        o = over ? o : up256(o + (bytes ? bytes : 1));
        return at;
    };
    L.ds = take(sizeof(DsDev));
    L.x32 = take(sizeof(float) * (size_t)n * ldx);
    L.xnorm = take(sizeof(float) * (size_t)n);
    L.mom = take(sizeof(float) * ((size_t)d + (d <= RRS_COV_MAX_D ? (size_t)d * d : 0) + 1));
    L.slots = take(sizeof(SlotDev) * (size_t)nq);
    L.gen = take(sizeof(TaskDev) * (size_t)nq * gen_per);
    L.hd = take(sizeof(TaskDev) * (size_t)nq * hd_per);
    L.pd = take(sizeof(TaskDev) * (size_t)nq * pd_per);
    L.arg = take(sizeof(int32_t) * (size_t)nq);
    L.z32 = take(sizeof(float) * (size_t)nq * ldx);
    L.poles = take(sizeof(float) * 2 * (size_t)nq * ldx);
    L.z64 = take(sizeof(double) * (size_t)nq * d);
    L.U = take(sizeof(float) * (size_t)nq * m * ldx);
    L.yz = take(sizeof(double) * (size_t)nq * m);
    L.res = take(sizeof(ResDev) * (size_t)nq * m);
    L.err = take(sizeof(int) * 2);
    L.total = over ? (size_t)RRS_NOALLOC_SCRATCH_BYTES + 1 : o;
    return L;
}

// Launch tables and per-query slots, written on the device (no host tables).
__global__ void k_noalloc_plan(DsDev* ds, const float* X32, const double* X64, const float* xnorm,
                               const float* center, const float* cov, const float* rc, int64_t n, int d,
                               int ldx, SlotDev* slots, TaskDev* gen, TaskDev* hd, TaskDev* pd, int32_t* arg,
                               int64_t nq, int kind, int m, int r, float alpha, uint64_t seed, const void* Z,
                               int zdtype, double* depth_out, int64_t* count_out, int gen_per, int hd_per,
                               int hd_size, int pd_per, int pd_size)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0) {
        DsDev D{};
        D.X32 = X32;
        D.X64 = X64;
        D.xnorm = xnorm;
        D.Xbf = nullptr;
        D.n = n;
        D.d = d;
        D.ldx = ldx;
        D.kp = 0;
        D.center = center;
        D.cov = cov;
        D.rc = *rc;
        *ds = D;
    }
    if (q >= nq) return;
    SlotDev S{};
    S.ds = 0;
    S.kind = kind;
    S.m = m;
    S.r = r;
    S.alpha = alpha;
    S.d = d;
    S.ldx = ldx;
    S.zdtype = zdtype;
    S.seed = seed;
    S.qctr = q;
    S.uoff = q * (int64_t)m * ldx;
    S.roff = q * (int64_t)m;
    S.zoff32 = q * (int64_t)ldx;
    S.zoff64 = q * (int64_t)d;
    S.zsrc = (const char*)Z + (size_t)q * d * (zdtype == 0 ? 4 : 8);
    S.depth_out = depth_out + q;
    S.count_out = count_out ? count_out + q : nullptr;
    S.best_out = nullptr;
    S.choice_out = nullptr;
    slots[q] = S;
    for (int t = 0; t < gen_per; ++t) {
        const int j0 = t * 128;
        gen[q * gen_per + t] = TaskDev{(int32_t)q, j0, m - j0 < 128 ? m - j0 : 128, 0};
    }
    if (kind == 0) {
        for (int t = 0; t < hd_per; ++t) {
            const int j0 = t * hd_size;
            hd[q * hd_per + t] = TaskDev{(int32_t)q, j0, m - j0 < hd_size ? m - j0 : hd_size, 0};
        }
    } else {
        for (int t = 0; t < pd_per; ++t) {
            const int j0 = t * pd_size;
            pd[q * pd_per + t] = TaskDev{(int32_t)q, j0, m - j0 < pd_size ? m - j0 : pd_size, 0};
        }
    }
    arg[q] = (int32_t)q;
}

}  // namespace

extern "C" rrs_status rrs_depth_noalloc(const void* X, int64_t n, int32_t d, int32_t dtype, const void* Z,
                                        int64_t n_queries, int32_t kind, int32_t n_dirs, int32_t n_refinements,
                                        double cap_shrink, uint64_t seed, double* depth_out, int64_t* count_out,
                                        void* stream)
{
    if (!X || n < 1 || d < 1 || d > 1024 || n_queries < 0 || (n_queries > 0 && (!Z || !depth_out)))
        return noalloc_fail(RRS_ERR_INVALID_ARG, "bad pointers or sizes");
    if (dtype != RRS_F32 && dtype != RRS_F64) return noalloc_fail(RRS_ERR_INVALID_ARG, "unknown dtype");
    if (kind < 0 || kind > 2) return noalloc_fail(RRS_ERR_INVALID_ARG, "unknown depth kind");
    if (n_refinements < 1 || n_dirs < n_refinements)
        return noalloc_fail(RRS_ERR_INVALID_ARG, "need n_dirs >= n_refinements >= 1");
    if (!(cap_shrink > 0.0) || cap_shrink > 1.0) return noalloc_fail(RRS_ERR_INVALID_ARG, "cap_shrink not in (0, 1]");
    if (n_queries == 0) return RRS_OK;
    const int ldx = padded_stride(d);
    const int m = (int)(((int64_t)n_dirs + n_refinements - 1) / n_refinements);
    // n, n_queries and n_queries * m are at most the scratch size (2^25 bytes) and ldx is at most
    // 1,028, so no size product of layout() can wrap a 64-bit size_t
    const int64_t cap = (int64_t)RRS_NOALLOC_SCRATCH_BYTES;
    if (n_queries > 0x7FFFFFFF || n_queries > cap || n > cap || (int64_t)n_queries * m > cap)
        return noalloc_fail(RRS_ERR_BUDGET,
                            "n = %lld, n_queries = %lld and n_dirs = %d need more than the %zu bytes of the "
                            "static scratch of rrs_depth_noalloc",
                            (long long)n, (long long)n_queries, n_dirs, (size_t)RRS_NOALLOC_SCRATCH_BYTES);
    if (kind == RRS_HALFSPACE && ldx > 440)
        return noalloc_fail(RRS_ERR_UNSUPPORTED, "d=%d too large for the FP32 halfspace kernel", d);
    int G = 0, pd_variant = 0;
    size_t pd_smem = 0;
    if (kind != RRS_HALFSPACE) {
        if (n > PDAP_MAX_N) return noalloc_fail(RRS_ERR_UNSUPPORTED, "n too large");
        // keys formed inside the selection kernel (no k_keys scratch here): resident when they fit
        // shared memory, else recomputed at every pass
        int Gr = pdap_max_group((int)n, ldx, m, d);
        if (Gr) {
            G = Gr;
            pd_variant = pdap_dp4_class(d);
            pd_smem = pdap_smem_bytes((int)n, G, ldx);
        } else {
            G = PDAP_STREAM_GROUP;
            pd_variant = pdap_dp4_class(d) | PDAP_STREAM;
            pd_smem = pdap_smem_bytes((int)n, G, ldx, true);
        }
    }
    const int gen_per = (m + 127) / 128;
    const int hd_tasks = (m + 63) / 64;
    const int hd_size = (m + hd_tasks - 1) / hd_tasks;
    const int hd_per = kind == RRS_HALFSPACE ? (m + hd_size - 1) / hd_size : 0;
    const int pd_per = kind == RRS_HALFSPACE ? 0 : (m + G - 1) / G;
    if ((int64_t)n_queries * gen_per > 0x7FFFFFFF || (int64_t)n_queries * hd_per > 0x7FFFFFFF ||
        (int64_t)n_queries * pd_per > 0x7FFFFFFF)
        return noalloc_fail(RRS_ERR_UNSUPPORTED, "too many queries");
    const Layout L = layout(n, ldx, d, n_queries, m, gen_per, hd_per, pd_per);
    if (L.total > (size_t)RRS_NOALLOC_SCRATCH_BYTES)
        return noalloc_fail(RRS_ERR_BUDGET,
                            "this call needs %zu bytes of working memory; the static scratch of "
                            "rrs_depth_noalloc holds %zu bytes",
                            L.total, (size_t)RRS_NOALLOC_SCRATCH_BYTES);

    void* base = nullptr;
    rrs_status s = scratch_address(&base);
    if (s != RRS_OK) return s;
    char* B = (char*)base;
    cudaStream_t st = (cudaStream_t)stream;
    DsDev* ds = (DsDev*)(B + L.ds);
    float* X32 = (float*)(B + L.x32);
    float* xnorm = (float*)(B + L.xnorm);
    SlotDev* slots = (SlotDev*)(B + L.slots);
    TaskDev* gen = (TaskDev*)(B + L.gen);
    TaskDev* hd = (TaskDev*)(B + L.hd);
    TaskDev* pd = (TaskDev*)(B + L.pd);
    int32_t* arg = (int32_t*)(B + L.arg);
    float* z32 = (float*)(B + L.z32);
    float* poles = (float*)(B + L.poles);
    double* z64 = (double*)(B + L.z64);
    float* U = (float*)(B + L.U);
    double* yz = (double*)(B + L.yz);
    ResDev* res = (ResDev*)(B + L.res);
    int* err = (int*)(B + L.err);   // [0] input check, [1] kernel error flags

#define NA_TRY(expr)                                                                                 \
    do {                                                                                             \
        cudaError_t _e = (expr);                                                                     \
        if (_e != cudaSuccess) {                                                                     \
            cudaGetLastError();                                                                      \
            return noalloc_fail(RRS_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e));              \
        }                                                                                            \
    } while (0)

    NA_TRY(cudaMemsetAsync(err, 0, 2 * sizeof(int), st));
    const double* X64 = dtype == RRS_F64 ? (const double*)X : nullptr;
    NA_TRY(launch_convert_dataset(X, dtype, n, d, ldx, X32, nullptr, xnorm, err, st));
    NA_TRY(launch_check_finite(Z, dtype, n_queries * d, err, st));
    float* center = (float*)(B + L.mom);
    float* cov = d <= RRS_COV_MAX_D ? center + d : nullptr;
    float* rc = center + d + (d <= RRS_COV_MAX_D ? (size_t)d * d : 0);
    NA_TRY(launch_moments(X32, n, d, ldx, center, cov, rc, st));
    const int nt = 128;
    k_noalloc_plan<<<(unsigned)((n_queries + nt - 1) / nt), nt, 0, st>>>(
        ds, X32, X64, xnorm, center, cov, rc, n, d, ldx, slots, gen, hd, pd, arg, n_queries, kind, m, n_refinements,
        (float)cap_shrink, seed, Z, dtype, depth_out, count_out, gen_per, hd_per, hd_size, pd_per, G);
    NA_TRY(cudaGetLastError());
    int bad = 0;
    NA_TRY(cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    if (bad) return noalloc_fail(RRS_ERR_INVALID_ARG, "X or Z holds a non-finite value or one of magnitude >= 2^64");

    const int nq = (int)n_queries;
    NA_TRY(launch_prep(slots, nq, ds, z32, z64, poles, st));
    const int64_t T = (int64_t)n_queries * ldx;
    for (int l = 0; l < n_refinements; ++l) {
        float* cur = poles + (l & 1) * T;
        float* nxt = poles + ((l + 1) & 1) * T;
        NA_TRY(launch_gen(gen, nq * gen_per, slots, cur, z64, U, yz, l, ldx, st));
        if (kind == RRS_HALFSPACE)
            NA_TRY(launch_hd_simt(hd, nq * hd_per, ldx, slots, ds, U, yz, z64, res, nullptr, err + 1, st));
        else
            NA_TRY(launch_pdap(pd, nq * pd_per, pd_smem, G, pd_variant, slots, ds, U, yz, res, err + 1, st));
        NA_TRY(launch_argmin(slots, arg, nq, U, res, cur, nxt, l, 0, st));
    }
    int flags = 0;
    NA_TRY(cudaMemcpyAsync(&flags, err + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    if (flags) return noalloc_fail(RRS_ERR_INTERNAL, "device-side error flags 0x%x", flags);
#undef NA_TRY
    return RRS_OK;
}
