// RRS round kernels for sm_103a: direction generation (Alg. S1/S4), halfspace
// counts on the CUDA cores with an exact near-tie recheck (Sec. 2, D_H),
// projection / asymmetric projection depth by bucket selection (Sec. 2, D_P
// and D_AP), and the round minimum with the pole update (Alg. 1 steps 4-6).
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "rrs_device.cuh"
#include "rrs_internal.h"

namespace rrs {

using namespace rrsdev;

__host__ __device__ float band_gamma_fp32(int d)
{
    // |fl32 dot - exact| <= gamma_d sum|u x| (gamma_d ~ d 2^-24), plus one rounding of x to FP32
    // (FP64 inputs), of y_z to FP32 and of the final difference; twice that sum for slack.
    return (float)((double)(d + 4) * 0x1p-23);
}

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

__global__ void k_gen(const TaskDev* __restrict__ tasks, const SlotDev* __restrict__ slots,
                      const float* __restrict__ poles, const double* __restrict__ z64, float* __restrict__ U,
                      double* __restrict__ yz, int round0)
{
    const TaskDev T = tasks[blockIdx.x];
    const int jl = threadIdx.x;
    if (jl >= T.nj) return;
    const SlotDev& S = slots[T.slot];
    const int j = T.j0 + jl;
    float* u = U + S.uoff + (int64_t)j * S.ldx;
    const float ap = alpha_power(S.alpha, round0);
    stream_direction(S.seed, (uint32_t)S.qctr, (uint32_t)round0, (uint32_t)j, S.d, ap, poles + S.zoff32, u, 1);
    for (int l = S.d; l < S.ldx; ++l) u[l] = 0.0f;
    double acc = 0.0;
    const double* z = z64 + S.zoff64;
    for (int l = 0; l < S.d; ++l) acc = __fma_rn((double)u[l], z[l], acc);
    yz[S.roff + j] = acc;
}

cudaError_t launch_gen(const TaskDev* tasks, int ntasks, const SlotDev* slots, const float* poles_cur,
                       const double* z64, float* U, double* yz, int round0, cudaStream_t st)
{
    if (ntasks <= 0) return cudaSuccess;
    k_gen<<<ntasks, 128, 0, st>>>(tasks, slots, poles_cur, z64, U, yz, round0);
    return cudaGetLastError();
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
        if (e != cudaSuccess) return e;
    }
    k_hd_simt<<<ntasks, HD_NT, smem, st>>>(tasks, slots, ds, U, yz, z64, res, band_out, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// projection / asymmetric projection depth: keys in shared memory, exact
// order statistics by bucket selection
// ---------------------------------------------------------------------------

constexpr int PD_NT = 512;
constexpr int PD_NW = PD_NT / 32;
constexpr int PD_NB = 2048;    // histogram bins
constexpr int PD_CAP = 512;    // candidates gathered for the final ranking
constexpr int PD_MAXG = 8;

struct SelShared {
    float fred[PD_NW * 2];
    int ired[PD_NW];
    int b1, b2, c1, c2;        // bins of the two ranks and elements below them
    int nbuf;
    float v1, v2;
};

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fminf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}
__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ void block_minmax(float& lo, float& hi, SelShared* sh)
{
    lo = warp_min(lo);
    hi = warp_max(hi);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        sh->fred[w] = lo;
        sh->fred[PD_NW + w] = hi;
    }
    __syncthreads();
    lo = sh->fred[0];
    hi = sh->fred[PD_NW];
    for (int i = 1; i < PD_NW; ++i) {
        lo = fminf(lo, sh->fred[i]);
        hi = fmaxf(hi, sh->fred[PD_NW + i]);
    }
}

__device__ int block_sum(int v, SelShared* sh)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh->ired[w] = v;
    __syncthreads();
    int s = 0;
    for (int i = 0; i < PD_NW; ++i) s += sh->ired[i];
    return s;
}

__device__ __forceinline__ int bucket_of(float a, float lo, float scale)
{
    const int b = __float2int_rz(__fmul_rn(__fsub_rn(a, lo), scale));
    return b < PD_NB - 1 ? b : PD_NB - 1;
}

// Values of 0-based ranks q1 <= q2 among the L values f(0..L-1), all of which
// lie in [lo, hi].  Exact: bucket indices are a monotone function of the
// value, so every bucket holds a contiguous run of ranks.
template <class F>
__device__ void select_ranks(F f, int L, int q1, int q2, float lo, float hi, unsigned* hist, float* buf,
                             SelShared* sh, float& v1, float& v2, int* err)
{
    const int tid = threadIdx.x;
    int below = 0;
    for (int iter = 0; iter < 24; ++iter) {
        if (!(lo < hi)) {
            v1 = v2 = lo;
            return;
        }
        float scale = __fdiv_rn((float)PD_NB, __fsub_rn(hi, lo));
        if (!(scale <= FLT_MAX)) scale = FLT_MAX;
        for (int b = tid; b < PD_NB; b += PD_NT) hist[b] = 0u;
        __syncthreads();
        for (int i = tid; i < L; i += PD_NT) {
            const float a = f(i);
            if (a >= lo && a <= hi) atomicAdd(&hist[bucket_of(a, lo, scale)], 1u);
        }
        __syncthreads();
        // exclusive scan of the histogram; thread t owns bins [4t, 4t+4)
        const int r1 = q1 - below, r2 = q2 - below;
        {
            unsigned h0 = hist[4 * tid], h1 = hist[4 * tid + 1], h2 = hist[4 * tid + 2], h3 = hist[4 * tid + 3];
            int own = (int)(h0 + h1 + h2 + h3);
            int incl = own;
            const int lane = tid & 31, w = tid >> 5;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) sh->ired[w] = incl;
            __syncthreads();
            int base = 0;
            for (int i = 0; i < w; ++i) base += sh->ired[i];
            int c = base + incl - own;
            const unsigned hh[4] = {h0, h1, h2, h3};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int h = (int)hh[k];
                if (h > 0) {
                    if (c <= r1 && r1 < c + h) { sh->b1 = 4 * tid + k; sh->c1 = c; }
                    if (c <= r2 && r2 < c + h) { sh->b2 = 4 * tid + k; sh->c2 = c; }
                }
                c += h;
            }
            if (tid == 0) sh->nbuf = 0;
        }
        __syncthreads();
        const int b1 = sh->b1, b2 = sh->b2, c1 = sh->c1, c2 = sh->c2;
        const int cnt = c2 + (int)hist[b2] - c1;
        if (cnt <= PD_CAP) {
            for (int i = tid; i < L; i += PD_NT) {
                const float a = f(i);
                if (a >= lo && a <= hi) {
                    const int b = bucket_of(a, lo, scale);
                    if (b >= b1 && b <= b2) buf[atomicAdd(&sh->nbuf, 1)] = a;
                }
            }
            __syncthreads();
            const int s1 = r1 - c1, s2 = r2 - c1;
            for (int t = tid; t < cnt; t += PD_NT) {
                const float v = buf[t];
                int nlt = 0, nle = 0;
                for (int s = 0; s < cnt; ++s) {
                    const float w2 = buf[s];
                    nlt += (w2 < v);
                    nle += (w2 <= v);
                }
                if (nlt <= s1 && s1 < nle) sh->v1 = v;
                if (nlt <= s2 && s2 < nle) sh->v2 = v;
            }
            __syncthreads();
            v1 = sh->v1;
            v2 = sh->v2;
            __syncthreads();
            return;
        }
        // too many candidates: narrow the range to buckets b1..b2 and repeat
        float nlo = FLT_MAX, nhi = -FLT_MAX;
        for (int i = tid; i < L; i += PD_NT) {
            const float a = f(i);
            if (a >= lo && a <= hi) {
                const int b = bucket_of(a, lo, scale);
                if (b >= b1 && b <= b2) {
                    nlo = fminf(nlo, a);
                    nhi = fmaxf(nhi, a);
                }
            }
        }
        block_minmax(nlo, nhi, sh);
        below += c1;
        lo = nlo;
        hi = nhi;
        __syncthreads();
    }
    if (tid == 0) atomicOr(err, ERR_SELECT_ITER);
    v1 = v2 = __int_as_float(0x7FC00000);
}

size_t pdap_smem_bytes(int n, int group, int ldx)
{
    return sizeof(float) * ((((size_t)group * n + 3) & ~(size_t)3) + (size_t)group * ldx + PD_CAP) +
           sizeof(unsigned) * PD_NB + sizeof(float) * 2 * PD_MAXG + 64;
}

int pdap_max_group(int n, int ldx, int m)
{
    // prefer two resident CTAs per SM (up to 110 KB each), else one (227 KB)
    const size_t two = 110 * 1024, one = 227 * 1024;
    int best = 0;
    for (int g = 1; g <= PD_MAXG && g <= m; ++g)
        if (pdap_smem_bytes(n, g, ldx) <= two) best = g;
    if (best == 0 && pdap_smem_bytes(n, 1, ldx) <= one) best = 1;
    return best;
}

__global__ void __launch_bounds__(PD_NT) k_pdap(const TaskDev* __restrict__ tasks, const SlotDev* __restrict__ slots,
                                                const DsDev* __restrict__ dsets, const float* __restrict__ U,
                                                const float* __restrict__ z32, ResDev* __restrict__ res, int* err)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ SelShared sh;
    const TaskDev T = tasks[blockIdx.x];
    const SlotDev& S = slots[T.slot];
    const DsDev D = dsets[S.ds];
    const int n = (int)D.n, ldx = D.ldx, d = D.d, dp4 = (d + 3) & ~3;
    const int G = T.nj;
    float* keys = sm;                                // G x n (region padded to a float4 multiple)
    float* uS = keys + (((size_t)G * n + 3) & ~(size_t)3);   // G x ldx, 16-byte aligned
    float* buf = uS + (size_t)G * ldx;               // PD_CAP
    unsigned* hist = reinterpret_cast<unsigned*>(buf + PD_CAP);   // PD_NB
    float* mm = reinterpret_cast<float*>(hist + PD_NB);           // 2 x PD_MAXG
    const int tid = threadIdx.x;

    for (int e = tid; e < G * ldx; e += PD_NT) uS[e] = U[S.uoff + (int64_t)T.j0 * ldx + e];
    __syncthreads();

    float lo[PD_MAXG], hi[PD_MAXG];
#pragma unroll
    for (int g = 0; g < PD_MAXG; ++g) {
        lo[g] = FLT_MAX;
        hi[g] = -FLT_MAX;
    }
    for (int i = tid; i < n; i += PD_NT) {
        const float4* xr = reinterpret_cast<const float4*>(D.X32 + (int64_t)i * ldx);
        float acc[PD_MAXG];
#pragma unroll
        for (int g = 0; g < PD_MAXG; ++g) acc[g] = 0.0f;
        for (int l = 0; l < dp4; l += 4) {
            const float4 x = xr[l >> 2];
#pragma unroll
            for (int g = 0; g < PD_MAXG; ++g) {
                if (g < G) {
                    const float4 u = *reinterpret_cast<const float4*>(uS + g * ldx + l);
                    acc[g] = fmaf(u.x, x.x, acc[g]);
                    acc[g] = fmaf(u.y, x.y, acc[g]);
                    acc[g] = fmaf(u.z, x.z, acc[g]);
                    acc[g] = fmaf(u.w, x.w, acc[g]);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < PD_MAXG; ++g) {
            if (g < G) {
                keys[(size_t)g * n + i] = acc[g];
                lo[g] = fminf(lo[g], acc[g]);
                hi[g] = fmaxf(hi[g], acc[g]);
            }
        }
    }
#pragma unroll
    for (int g = 0; g < PD_MAXG; ++g) {
        if (g < G) {
            block_minmax(lo[g], hi[g], &sh);
            if (tid == 0) {
                mm[2 * g] = lo[g];
                mm[2 * g + 1] = hi[g];
            }
        }
    }
    __syncthreads();

    const int k1 = (n - 1) / 2, k2 = n / 2;
    for (int g = 0; g < G; ++g) {
        const float* y = keys + (size_t)g * n;
        const float ylo = mm[2 * g], yhi = mm[2 * g + 1];
        float m1, m2;
        select_ranks([&](int i) { return y[i]; }, n, k1, k2, ylo, yhi, hist, buf, &sh, m1, m2, err);
        const double med = ((double)m1 + (double)m2) * 0.5;
        // y_z with exactly the arithmetic of the data projections, so a query equal to a data
        // point projects to the same FP32 value as that point
        float yzf = 0.0f;
        {
            const float* zr = z32 + S.zoff32;
            for (int l = 0; l < dp4; l += 4) {
                yzf = fmaf(uS[g * ldx + l + 0], zr[l + 0], yzf);
                yzf = fmaf(uS[g * ldx + l + 1], zr[l + 1], yzf);
                yzf = fmaf(uS[g * ldx + l + 2], zr[l + 2], yzf);
                yzf = fmaf(uS[g * ldx + l + 3], zr[l + 3], yzf);
            }
        }
        const double yzv = (double)yzf;
        double depth;
        if (S.kind == 1) {
            auto dev = [&](int i) { return __double2float_rn(fabs((double)y[i] - med)); };
            const float dhi = fmaxf(__double2float_rn(fabs((double)ylo - med)), __double2float_rn(fabs((double)yhi - med)));
            float a1, a2;
            select_ranks(dev, n, k1, k2, 0.0f, dhi, hist, buf, &sh, a1, a2, err);
            const double mad = ((double)a1 + (double)a2) * 0.5;
            const double num = fabs(yzv - med);
            depth = (mad == 0.0) ? (num == 0.0 ? 1.0 : 0.0) : 1.0 / (1.0 + num / mad);
        } else {
            int cpos = 0;
            for (int i = tid; i < n; i += PD_NT) cpos += ((double)y[i] > med);
            const int npos = block_sum(cpos, &sh);
            double madp = 0.0;
            if (npos > 0) {
                const int base = n - npos;
                float p1, p2;
                select_ranks([&](int i) { return y[i]; }, n, base + (npos - 1) / 2, base + npos / 2, ylo, yhi, hist,
                             buf, &sh, p1, p2, err);
                madp = (((double)p1 - med) + ((double)p2 - med)) * 0.5;
            }
            const double num = yzv - med > 0.0 ? yzv - med : 0.0;
            depth = (madp == 0.0) ? (num == 0.0 ? 1.0 : 0.0) : 1.0 / (1.0 + num / madp);
        }
        if (tid == 0) res[S.roff + T.j0 + g] = ResDev{depth, -1};
        __syncthreads();
    }
}

cudaError_t launch_pdap(const TaskDev* tasks, int ntasks, size_t smem, const SlotDev* slots, const DsDev* ds,
                        const float* U, const float* z32, ResDev* res, int* err, cudaStream_t st)
{
    if (ntasks <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_pdap, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_pdap<<<ntasks, PD_NT, smem, st>>>(tasks, slots, ds, U, z32, res, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// round minimum, strict update of D_min and of the pole (Alg. 1 steps 4-6)
// ---------------------------------------------------------------------------

__global__ void k_argmin(SlotDev* __restrict__ slots, const int32_t* __restrict__ slot_list, int nlist,
                         const float* __restrict__ U, const ResDev* __restrict__ res, const float* __restrict__ poles_cur,
                         float* __restrict__ poles_next, int round0)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nlist) return;
    SlotDev& S = slots[slot_list[w]];
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
    }
}

cudaError_t launch_argmin(SlotDev* slots, const int32_t* slot_list, int nlist, const float* U, const ResDev* res,
                          const float* poles_cur, float* poles_next, int round0, int last_round, cudaStream_t st)
{
    if (nlist <= 0) return cudaSuccess;
    const int nt = 256;
    const int nb = (nlist * 32 + nt - 1) / nt;
    (void)last_round;
    k_argmin<<<nb, nt, 0, st>>>(slots, slot_list, nlist, U, res, poles_cur, poles_next, round0);
    return cudaGetLastError();
}

}  // namespace rrs
