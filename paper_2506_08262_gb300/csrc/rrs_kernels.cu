// RRS round kernels for sm_103a: direction generation (Alg. S1/S4), halfspace
// counts on the CUDA cores with an exact near-tie recheck (Sec. 2, D_H), and
// the round minimum with the pole update (Alg. 1 steps 4-6).  The D_P / D_AP
// selection kernel lives in pdap.cu.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "rrs_device.cuh"
#include "rrs_internal.h"

namespace rrs {

using namespace rrsdev;


// ---------------------------------------------------------------------------
// dataset and query preparation
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_convert_dataset(const T* __restrict__ X, int64_t n, int d, int ldx, float* __restrict__ X32,
                                  double* __restrict__ X64, float* __restrict__ xnorm, int* bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T* row = X + i * d;
    double s = 0.0;
    int isbad = 0;
    for (int l = 0; l < ldx; ++l) {
        if (l < d) {
            const double v = (double)row[l];
            if (!(fabs(v) < 1.8446744073709552e19)) isbad = 1;  // non-finite or |v| >= 2^64
            s = __fma_rn(v, v, s);
            X32[i * ldx + l] = (float)v;
            if (X64) X64[i * d + l] = v;
        } else {
            X32[i * ldx + l] = 0.0f;
        }
    }
    xnorm[i] = __double2float_ru(__dsqrt_ru(s) * (1.0 + 1e-12));
    if (isbad) atomicOr(bad, 1);
}

cudaError_t launch_convert_dataset(const void* X, int dtype, int64_t n, int d, int ldx, float* X32, double* X64,
                                   float* xnorm, int* bad, cudaStream_t st)
{
    const int nt = 128;
    const int64_t nb = (n + nt - 1) / nt;
    if (dtype == 0)
        k_convert_dataset<float><<<(unsigned)nb, nt, 0, st>>>((const float*)X, n, d, ldx, X32, X64, xnorm, bad);
    else
        k_convert_dataset<double><<<(unsigned)nb, nt, 0, st>>>((const double*)X, n, d, ldx, X32, X64, xnorm, bad);
    return cudaGetLastError();
}

// One thread per (row, 16-byte chunk) of the tiled copy, rows beyond n zero.
__global__ void k_tile_rows(const float4* __restrict__ X32, int64_t n, int c4, int64_t total, float4* __restrict__ Xt)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t lane = e & 31, rest = e >> 5;
    const int64_t c = rest % c4, tile = rest / c4;
    const int64_t i = tile * 32 + lane;
    Xt[e] = i < n ? X32[i * c4 + c] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

size_t tile_rows_floats(int64_t n, int ldx)
{
    return (size_t)((n + 31) / 32) * 32 * (size_t)ldx;
}

cudaError_t launch_tile_rows(const float* X32, int64_t n, int ldx, float* Xt, cudaStream_t st)
{
    const int64_t total = (int64_t)(tile_rows_floats(n, ldx) / 4);
    const int nt = 256;
    k_tile_rows<<<(unsigned)((total + nt - 1) / nt), nt, 0, st>>>((const float4*)X32, n, ldx / 4, total, (float4*)Xt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// data moments (range heuristics of the selection kernel only; no result
// depends on their accuracy)
// ---------------------------------------------------------------------------

__global__ void k_center(const float* __restrict__ X32, int64_t n, int ldx, float* __restrict__ center)
{
    const int a = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)X32[i * ldx + a];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) center[a] = (float)(red[0] / (double)n);
}

__global__ void k_cov(const float* __restrict__ X32, int64_t n, int d, int ldx, const float* __restrict__ center,
                      float* __restrict__ cov)
{
    const int a = blockIdx.x / d, b = blockIdx.x % d;
    if (b < a) return;
    const float ca = center[a], cb = center[b];
    float s = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fmaf(X32[i * ldx + a] - ca, X32[i * ldx + b] - cb, s);
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float v = red[0] / (float)n;
        cov[a * d + b] = v;
        cov[b * d + a] = v;
    }
}

__global__ void k_radius(const float* __restrict__ X32, int64_t n, int d, int ldx, const float* __restrict__ center,
                         float* rc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int l = 0; l < d; ++l) {
        const double v = (double)X32[i * ldx + l] - (double)center[l];
        s = __fma_rn(v, v, s);
    }
    const float r = __double2float_ru(__dsqrt_ru(s) * (1.0 + 1e-9));
    atomicMax((int*)rc, __float_as_int(r));   // non-negative floats order like their bit patterns
}

cudaError_t launch_moments(const float* X32, int64_t n, int d, int ldx, float* center, float* cov, float* rc_out,
                           cudaStream_t st)
{
    k_center<<<d, 256, 0, st>>>(X32, n, ldx, center);
    if (cov) k_cov<<<d * d, 256, 0, st>>>(X32, n, d, ldx, center, cov);
    cudaError_t e = cudaMemsetAsync(rc_out, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    k_radius<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(X32, n, d, ldx, center, rc_out);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_check_finite(const T* __restrict__ Z, int64_t count, int* bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        if (!(fabs((double)Z[i]) < 1.8446744073709552e19)) atomicOr(bad, 1);
}

cudaError_t launch_check_finite(const void* Z, int dtype, int64_t count, int* bad, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const int nt = 256;
    int64_t nb = (count + nt - 1) / nt;
    if (nb > 4096) nb = 4096;
    if (dtype == 0) k_check_finite<float><<<(unsigned)nb, nt, 0, st>>>((const float*)Z, count, bad);
    else k_check_finite<double><<<(unsigned)nb, nt, 0, st>>>((const double*)Z, count, bad);
    return cudaGetLastError();
}

__global__ void k_prep(SlotDev* slots, int nslots, const DsDev* ds, float* z32, double* z64, float* poles)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    SlotDev& S = slots[s];
    const int d = S.d, ldx = S.ldx;
    double acc = 0.0;
    for (int l = 0; l < ldx; ++l) {
        double v = 0.0;
        if (l < d) {
            v = S.zdtype == 0 ? (double)((const float*)S.zsrc)[l] : ((const double*)S.zsrc)[l];
            z64[S.zoff64 + l] = v;
            acc = __fma_rn(v, v, acc);
        }
        z32[S.zoff32 + l] = (float)v;
        poles[S.zoff32 + l] = (l == 0) ? 1.0f : 0.0f;
    }
    S.znorm = __double2float_ru(__dsqrt_ru(acc) * (1.0 + 1e-12));
    S.dmin = 1.0;
    S.cmin = ds[S.ds].n;
    S.best = -1;
}

cudaError_t launch_prep(const SlotDev* slots, int nslots, const DsDev* ds, float* z32, double* z64, float* poles,
                        cudaStream_t st)
{
    if (nslots <= 0) return cudaSuccess;
    const int nt = 128;
    k_prep<<<(nslots + nt - 1) / nt, nt, 0, st>>>((SlotDev*)slots, nslots, ds, z32, z64, poles);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// direction generation: one thread per (slot, direction)
// ---------------------------------------------------------------------------

// One thread per direction of one query (a task never spans queries).  With d <= stage_d the CTA builds
// its directions in shared memory, transposed (element i of thread t at i * GEN_STRIDE + t: the passes
// of the generator, the same arithmetic in the same order, touch consecutive banks), and then writes
// the rows out whole, coalesced; larger d builds each row in place in U.
constexpr int GEN_NT = 128, GEN_STRIDE = GEN_NT + 1;
constexpr size_t GEN_STAGE_MAX = 96 * 1024;

__global__ void __launch_bounds__(GEN_NT) k_gen(const TaskDev* __restrict__ tasks, const SlotDev* __restrict__ slots,
                                                const float* __restrict__ poles, const float* __restrict__ poles1,
                                                const double* __restrict__ z64, float* __restrict__ U,
                                                double* __restrict__ yz, int round0, int stage_d)
{
    extern __shared__ float gstage[];
    const TaskDev T = tasks[blockIdx.x];
    const int jl = threadIdx.x;
    const SlotDev& S = slots[T.slot];
    // launch-wide round, or (round0 < 0) the slot's own round with its pole buffer by parity
    const int rnd = round0 >= 0 ? round0 : S.round;
    const float* pcur = round0 >= 0 ? poles : ((rnd & 1) ? poles1 : poles);
    const int j = T.j0 + jl;
    const float ap = alpha_power(S.alpha, rnd);
    const double* z = z64 + S.zoff64;
    if (S.d > stage_d) {
        if (jl >= T.nj) return;
        float* u = U + S.uoff + (int64_t)j * S.ldx;
        stream_direction(S.seed, (uint32_t)S.qctr, (uint32_t)rnd, (uint32_t)j, S.d, ap, pcur + S.zoff32, u, 1);
        for (int l = S.d; l < S.ldx; ++l) u[l] = 0.0f;
        double acc = 0.0;
        for (int l = 0; l < S.d; ++l) acc = __fma_rn((double)u[l], z[l], acc);
        yz[S.roff + j] = acc;
        return;
    }
    if (jl < T.nj) {
        float* u = gstage + jl;
        stream_direction(S.seed, (uint32_t)S.qctr, (uint32_t)rnd, (uint32_t)j, S.d, ap, pcur + S.zoff32, u,
                         GEN_STRIDE);
        double acc = 0.0;
        for (int l = 0; l < S.d; ++l) acc = __fma_rn((double)u[l * GEN_STRIDE], z[l], acc);
        yz[S.roff + j] = acc;
    }
    __syncthreads();
    // rows j0 .. j0 + nj - 1 of this query are contiguous in U
    float* base = U + S.uoff + (int64_t)T.j0 * S.ldx;
    const int ldx = S.ldx, total = T.nj * ldx;
    for (int e = jl; e < total; e += GEN_NT) {
        const int r = e / ldx, l = e - r * ldx;
        base[e] = l < S.d ? gstage[l * GEN_STRIDE + r] : 0.0f;
    }
}

// directions of up to max_ldx dims are staged in shared memory (up to GEN_STAGE_MAX bytes)
static cudaError_t gen_launch(const TaskDev* tasks, int ntasks, const SlotDev* slots, const float* p0,
                              const float* p1, const double* z64, float* U, double* yz, int round0, int max_ldx,
                              cudaStream_t st)
{
    if (ntasks <= 0) return cudaSuccess;
    int stage_d = max_ldx;
    const size_t per_dim = sizeof(float) * GEN_STRIDE;
    if ((size_t)stage_d * per_dim > GEN_STAGE_MAX) stage_d = (int)(GEN_STAGE_MAX / per_dim);
    const size_t smem = (size_t)stage_d * per_dim;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
    }
    k_gen<<<ntasks, GEN_NT, smem, st>>>(tasks, slots, p0, p1, z64, U, yz, round0, stage_d);
    return cudaGetLastError();
}

cudaError_t launch_gen(const TaskDev* tasks, int ntasks, const SlotDev* slots, const float* poles_cur,
                       const double* z64, float* U, double* yz, int round0, int max_ldx, cudaStream_t st)
{
    return gen_launch(tasks, ntasks, slots, poles_cur, nullptr, z64, U, yz, round0, max_ldx, st);
}

cudaError_t launch_gen_slotround(const TaskDev* tasks, int ntasks, const SlotDev* slots, const float* poles0,
                                 const float* poles1, const double* z64, float* U, double* yz, int max_ldx,
                                 cudaStream_t st)
{
    return gen_launch(tasks, ntasks, slots, poles0, poles1, z64, U, yz, -1, max_ldx, st);
}

// y_z = u'z in FP64 for caller-supplied directions (debug path)
__global__ void k_yz_only(const TaskDev* __restrict__ tasks, const SlotDev* __restrict__ slots,
                          const double* __restrict__ z64, const float* __restrict__ U, double* __restrict__ yz)
{
    const TaskDev T = tasks[blockIdx.x];
    const int jl = threadIdx.x;
    if (jl >= T.nj) return;
    const SlotDev& S = slots[T.slot];
    const int j = T.j0 + jl;
    const float* u = U + S.uoff + (int64_t)j * S.ldx;
    double acc = 0.0;
    const double* z = z64 + S.zoff64;
    for (int l = 0; l < S.d; ++l) acc = __fma_rn((double)u[l], z[l], acc);
    yz[S.roff + j] = acc;
}

cudaError_t launch_yz_only(const TaskDev* tasks, int ntasks, const SlotDev* slots, const double* z64, const float* U,
                           double* yz, cudaStream_t st)
{
    if (ntasks <= 0) return cudaSuccess;
    k_yz_only<<<ntasks, 128, 0, st>>>(tasks, slots, z64, U, yz);
    return cudaGetLastError();
}

// caller-supplied directions (n_slots x m x d, dense) into the padded U rows
__global__ void k_scatter_dirs(const SlotDev* __restrict__ slots, int nslots, int m, int d, const float* __restrict__ Uin,
                               float* __restrict__ U)
{
    const int s = blockIdx.x;
    if (s >= nslots) return;
    const SlotDev& S = slots[s];
    for (int e = threadIdx.x; e < m * S.ldx; e += blockDim.x) {
        const int j = e / S.ldx, l = e - j * S.ldx;
        U[S.uoff + e] = (l < d) ? Uin[((int64_t)s * m + j) * d + l] : 0.0f;
    }
}

cudaError_t launch_scatter_dirs(const SlotDev* slots, int nslots, int m, int d, const float* Uin, float* U,
                                cudaStream_t st)
{
    if (nslots <= 0) return cudaSuccess;
    k_scatter_dirs<<<nslots, 128, 0, st>>>(slots, nslots, m, d, Uin, U);
    return cudaGetLastError();
}

__global__ void k_debug_dirs(uint64_t seed, int q, int round0, int m, int d, float alpha, const float* pole,
                             float* U)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    stream_direction(seed, (uint32_t)q, (uint32_t)round0, (uint32_t)j, d, alpha_power(alpha, round0), pole,
                     U + (int64_t)j * d, 1);
}

cudaError_t launch_debug_dirs(uint64_t seed, int q, int round0, int m, int d, float alpha, const float* pole,
                              float* U, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    k_debug_dirs<<<(m + 127) / 128, 128, 0, st>>>(seed, q, round0, m, d, alpha, pole, U);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// halfspace counts, FP32 SIMT projection + exact recheck of the near-tie band
// ---------------------------------------------------------------------------

constexpr int HD_NT = 256;
constexpr int HD_TJ = 64;   // directions per CTA
constexpr int HD_PC = 64;   // points per staged chunk

__global__ void __launch_bounds__(HD_NT) k_hd_simt(const TaskDev* __restrict__ tasks,
                                                   const SlotDev* __restrict__ slots, const DsDev* __restrict__ dsets,
                                                   const float* __restrict__ U, const double* __restrict__ yz,
                                                   const double* __restrict__ z64, ResDev* __restrict__ res,
                                                   int64_t* __restrict__ band_out, int* err)
{
    extern __shared__ __align__(16) float sm[];
    const TaskDev T = tasks[blockIdx.x];
    const SlotDev& S = slots[T.slot];
    const DsDev D = dsets[S.ds];
    const int ldx = D.ldx, d = D.d, dp4 = (d + 3) & ~3;
    const int64_t n = D.n;
    float* uS = sm;                       // HD_TJ x ldx
    float* xS = uS + HD_TJ * ldx;         // HD_PC x ldx
    float* xnS = xS + HD_PC * ldx;        // HD_PC
    float* yzS = xnS + HD_PC;             // HD_TJ
    const int tid = threadIdx.x;

    for (int e = tid; e < HD_TJ * ldx; e += HD_NT) {
        const int j = e / ldx;
        uS[e] = (j < T.nj) ? U[S.uoff + (int64_t)(T.j0 + j) * ldx + (e - j * ldx)] : 0.0f;
    }
    for (int j = tid; j < HD_TJ; j += HD_NT) yzS[j] = (j < T.nj) ? (float)yz[S.roff + T.j0 + j] : 0.0f;

    const float gamma = band_gamma_fp32(d);
    const float zn = S.znorm;
    const double* zrow = z64 + S.zoff64;
    const int dg = tid >> 4, pg = tid & 15;
    int lt[4] = {0, 0, 0, 0}, gt[4] = {0, 0, 0, 0};
    int nband = 0;

    for (int64_t i0 = 0; i0 < n; i0 += HD_PC) {
        __syncthreads();
        const int64_t rows = (n - i0 < HD_PC) ? (n - i0) : HD_PC;
        const float4* src = reinterpret_cast<const float4*>(D.X32 + i0 * ldx);
        float4* dst = reinterpret_cast<float4*>(xS);
        const int nv = HD_PC * ldx / 4, nvalid = (int)rows * ldx / 4;
        for (int e = tid; e < nv; e += HD_NT) dst[e] = (e < nvalid) ? src[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int p = tid; p < HD_PC; p += HD_NT) xnS[p] = (p < rows) ? D.xnorm[i0 + p] : 0.0f;
        __syncthreads();

        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[a][t] = 0.0f;
        for (int l = 0; l < dp4; l += 4) {
            float4 uv[4], xv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) uv[a] = *reinterpret_cast<const float4*>(uS + (dg * 4 + a) * ldx + l);
#pragma unroll
            for (int t = 0; t < 4; ++t) xv[t] = *reinterpret_cast<const float4*>(xS + (pg + 16 * t) * ldx + l);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    acc[a][t] = fmaf(uv[a].x, xv[t].x, acc[a][t]);
                    acc[a][t] = fmaf(uv[a].y, xv[t].y, acc[a][t]);
                    acc[a][t] = fmaf(uv[a].z, xv[t].z, acc[a][t]);
                    acc[a][t] = fmaf(uv[a].w, xv[t].w, acc[a][t]);
                }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int p = pg + 16 * t;
            if (p >= rows) continue;
            const float b = gamma * (xnS[p] + zn);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int j = dg * 4 + a;
                if (j >= T.nj) continue;
                const float tv = acc[a][t] - yzS[j];
                if (tv < -b) {
                    lt[a]++;
                } else if (tv > b) {
                    gt[a]++;
                } else {
                    const int64_t i = i0 + p;
                    int s;
                    if (D.X64) s = exact_sign<double>(uS + j * ldx, 1, D.X64 + i * d, zrow, d, err);
                    else s = exact_sign<float>(uS + j * ldx, 1, D.X32 + i * ldx, zrow, d, err);
                    lt[a] += (s < 0);
                    gt[a] += (s > 0);
                    nband++;
                }
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int o = 8; o >= 1; o >>= 1) {
            lt[a] += __shfl_xor_sync(0xFFFFFFFFu, lt[a], o);
            gt[a] += __shfl_xor_sync(0xFFFFFFFFu, gt[a], o);
        }
    }
    if (band_out) {
        // band points are counted per thread over its directions; one total per CTA task
        __shared__ int bsum;
        if (tid == 0) bsum = 0;
        __syncthreads();
        atomicAdd(&bsum, nband);
        __syncthreads();
        if (tid == 0) atomicAdd((unsigned long long*)&band_out[T.slot], (unsigned long long)bsum);
    }
    if (pg == 0) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int j = dg * 4 + a;
            if (j < T.nj) {
                const int64_t le = n - gt[a], ge = n - lt[a];
                const int64_t c = le < ge ? le : ge;
                res[S.roff + T.j0 + j] = ResDev{(double)c / (double)n, c};
            }
        }
    }
}

cudaError_t launch_hd_simt(const TaskDev* tasks, int ntasks, int max_ldx, const SlotDev* slots,
                               const DsDev* ds, const float* U, const double* yz, const double* z64, ResDev* res,
                               int64_t* band_out, int* err, cudaStream_t st)
{
    if (ntasks <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * ((size_t)(HD_TJ + HD_PC) * max_ldx + HD_PC + HD_TJ);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_hd_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
    }
    k_hd_simt<<<ntasks, HD_NT, smem, st>>>(tasks, slots, ds, U, yz, z64, res, band_out, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// round minimum, strict update of D_min and of the pole (Alg. 1 steps 4-6)
// ---------------------------------------------------------------------------

__global__ void k_argmin(SlotDev* __restrict__ slots, const int32_t* __restrict__ slot_list, int nlist,
                         const float* __restrict__ U, const ResDev* __restrict__ res, float* __restrict__ pa,
                         float* __restrict__ pb, int round_arg)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nlist) return;
    SlotDev& S = slots[slot_list[w]];
    // launch-wide round (pa = current poles, pb = next), or the slot's own round (pa even, pb odd)
    const int round0 = round_arg >= 0 ? round_arg : S.round;
    const float* poles_cur = round_arg >= 0 ? pa : ((round0 & 1) ? pb : pa);
    float* poles_next = round_arg >= 0 ? pb : ((round0 & 1) ? pa : pb);
    const bool hd = (S.kind == 0);
    // lowest (value, index) over the m directions
    double bv = INFINITY;
    int64_t bc = INT64_MAX;
    int bj = INT32_MAX;
    for (int j = lane; j < S.m; j += 32) {
        const ResDev r = res[S.roff + j];
        const bool better = hd ? (r.count < bc) : (r.depth < bv);
        if (better) {
            bv = r.depth;
            bc = r.count;
            bj = j;
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const double ov = __shfl_xor_sync(0xFFFFFFFFu, bv, o);
        const int64_t oc = __shfl_xor_sync(0xFFFFFFFFu, bc, o);
        const int oj = __shfl_xor_sync(0xFFFFFFFFu, bj, o);
        const bool better = hd ? (oc < bc || (oc == bc && oj < bj)) : (ov < bv || (ov == bv && oj < bj));
        if (better) {
            bv = ov;
            bc = oc;
            bj = oj;
        }
    }
    const bool take = hd ? (bc < S.cmin) : (bv < S.dmin);
    const float* src = take ? U + S.uoff + (int64_t)bj * S.ldx : poles_cur + S.zoff32;
    for (int l = lane; l < S.ldx; l += 32) poles_next[S.zoff32 + l] = src[l];
    if (lane == 0) {
        if (take) {
            S.dmin = bv;
            S.cmin = bc;
            S.best = round0 * S.m + bj;
        }
        if (S.choice_out) S.choice_out[round0] = take ? bj : -1;
        if (round0 == S.r - 1) {
            if (S.depth_out) S.depth_out[0] = S.dmin;
            if (S.count_out) S.count_out[0] = hd ? S.cmin : -1;
            if (S.best_out) S.best_out[0] = S.best;
        }
        if (round_arg < 0) S.round = round0 + 1;
    }
}

cudaError_t launch_argmin(SlotDev* slots, const int32_t* slot_list, int nlist, const float* U, const ResDev* res,
                          const float* poles_cur, float* poles_next, int round0, int last_round, cudaStream_t st)
{
    if (nlist <= 0) return cudaSuccess;
    const int nt = 256;
    const int nb = (nlist * 32 + nt - 1) / nt;
    (void)last_round;
    k_argmin<<<nb, nt, 0, st>>>(slots, slot_list, nlist, U, res, const_cast<float*>(poles_cur), poles_next, round0);
    return cudaGetLastError();
}

cudaError_t launch_argmin_slotround(SlotDev* slots, const int32_t* slot_list, int nlist, const float* U,
                                   const ResDev* res, float* poles0, float* poles1, cudaStream_t st)
{
    if (nlist <= 0) return cudaSuccess;
    const int nt = 256;
    const int nb = (nlist * 32 + nt - 1) / nt;
    k_argmin<<<nb, nt, 0, st>>>(slots, slot_list, nlist, U, res, poles0, poles1, -1);
    return cudaGetLastError();
}

}  // namespace rrs
