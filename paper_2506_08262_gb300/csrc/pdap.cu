// Projection depth D_P and asymmetric projection depth D_AP (Sec. 2) for a block
// of directions: y_i = u'x_i in FP32, exact order statistics (median, MAD,
// MAD_+) of the FP32 keys, depth in FP64 from those few values.
//
// One CTA handles G <= 4 directions of one query with the G*n keys resident in
// shared memory.  Selection is bucket based and exact:
//   pass A  project every point on the G directions, store the keys and add
//           each to a 2048-bucket histogram over [-R, R], R = max |x_i| (a bound
//           on every |u'x_i|), bucket = monotone FP32 map of the key;
//   pass C  gather the keys of the buckets holding the median ranks (and,
//           for D_AP, of the buckets expected to hold the MAD_+ ranks), then
//           rank them exactly;
//   D_P     histogram of |y - med| over [0, R + |med|], gather, rank (MAD).
// Bucket maps are monotone, so every bucket holds a contiguous run of ranks
// and the gathered keys contain the wanted order statistics.  When a bucket
// run holds more keys than the gather buffer, or the D_AP guess of the
// positive count was wrong, that direction falls back to an iterated bucket
// selection over its keys.  No per-element work uses FP64.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "rrs_internal.h"

namespace rrs {
namespace {

constexpr int NT = 512;
constexpr int NWARP = NT / 32;
constexpr int NB = 2048;     // buckets per direction
constexpr int CAP = 256;     // gathered keys per direction and target
constexpr int MAXG = 4;
constexpr int FB_NB = NB;    // fallback histogram (reuses the bucket area)
constexpr int FB_CAP = 512;  // fallback gather buffer (reuses the gather area; 2*CAP*G >= 512)

struct Ctl {
    int b_lo[MAXG][2], b_hi[MAXG][2];  // bucket runs: [0] median (or MAD), [1] MAD_+ guess
    int c_lo[MAXG][2];                 // keys below the run
    int cnt[MAXG][2];                  // keys in the run
    int fill[MAXG][2];                 // keys gathered so far
    int fb[MAXG];                      // 1: fall back for all statistics, 2: only MAD_+
    float lo_b[MAXG], sc_y[MAXG];      // bucket map of the keys: about (y - lo_b) * sc_y
    float off_y[MAXG];                 // -lo_b * sc_y (bucket_fma offset)
    float scale[MAXG];                 // sigma_u (or the radius) of each direction
    float cen[MAXG], sc_d[MAXG];       // bucket map of |y - med| (D_P)
    float v1[MAXG][2], v2[MAXG][2];    // selected order statistics
    float yz[MAXG];
    int nle[MAXG];                     // #(y <= m1)
    int npos[MAXG];                    // #(y > med), D_AP
    int red[NWARP];
    float fred[2 * NWARP];
    // generic fallback
    int g_b1, g_b2, g_c1, g_c2, g_n;
    float g_v1, g_v2;
};

__device__ __forceinline__ int bucket(float y, float lo, float scale)
{
    // (y - lo) * scale, rounded once, truncated: monotone in y
    const int b = __float2int_rz(__fmul_rn(__fsub_rn(y, lo), scale));
    return b < 0 ? 0 : (b > NB - 1 ? NB - 1 : b);
}

// Bucket of the pass maps: y*sc + off rounded once, truncated (negatives saturate to 0),
// clamped to the last bucket.  Monotone non-decreasing in y.
__device__ __forceinline__ int bucket_fma(float y, float sc, float off)
{
    const unsigned b = __float2uint_rz(__fmaf_rn(y, sc, off));
    return b < (unsigned)(NB - 1) ? (int)b : NB - 1;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}
__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fminf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

// Exclusive scan of h[0..NB) by the whole CTA; records the bucket holding
// rank ra and the one holding rank rb (ra <= rb), with the keys below each.
__device__ void find_buckets(const unsigned* h, int ra, int rb, Ctl& C, int& ba, int& ca, int& bb, int& cb)
{
    constexpr int PER = NB / NT;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int own = 0;
    unsigned v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = h[tid * PER + k];
        own += (int)v[k];
    }
    int incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) C.red[w] = incl;
    __syncthreads();
    int base = 0;
    for (int i = 0; i < w; ++i) base += C.red[i];
    int c = base + incl - own;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int hk = (int)v[k];
        if (hk > 0) {
            if (c <= ra && ra < c + hk) { C.g_b1 = tid * PER + k; C.g_c1 = c; }
            if (c <= rb && rb < c + hk) { C.g_b2 = tid * PER + k; C.g_c2 = c; }
        }
        c += hk;
    }
    __syncthreads();
    ba = C.g_b1;
    ca = C.g_c1;
    bb = C.g_b2;
    cb = C.g_c2;
    __syncthreads();
}

// Rank among buf[0..cnt): values of 0-based ranks s1 <= s2.
__device__ __forceinline__ void rank_pick(const float* buf, int cnt, int t, int s1, int s2, float& o1, float& o2)
{
    const float v = buf[t];
    int nlt = 0, nle = 0;
    for (int s = 0; s < cnt; ++s) {
        const float w2 = buf[s];
        nlt += (w2 < v);
        nle += (w2 <= v);
    }
    if (nlt <= s1 && s1 < nle) o1 = v;
    if (nlt <= s2 && s2 < nle) o2 = v;
}

// Generic exact selection over one direction's keys f(0..L-1), all in
// [lo, hi], by iterated bucketing (the fallback path).
template <class F>
__device__ void select_generic(F f, int L, int q1, int q2, float lo, float hi, unsigned* hist, float* buf, Ctl& C,
                               float& v1, float& v2, int* err)
{
    const int tid = threadIdx.x;
    int below = 0;
    for (int iter = 0; iter < 24; ++iter) {
        if (!(lo < hi)) {
            v1 = v2 = lo;
            return;
        }
        float scale = __fdiv_rn((float)FB_NB, __fsub_rn(hi, lo));
        if (!(scale <= FLT_MAX)) scale = FLT_MAX;
        for (int b = tid; b < FB_NB; b += NT) hist[b] = 0u;
        __syncthreads();
        for (int i = tid; i < L; i += NT) {
            const float a = f(i);
            if (a >= lo && a <= hi) atomicAdd(&hist[bucket(a, lo, scale)], 1u);
        }
        __syncthreads();
        int b1, c1, b2, c2;
        find_buckets(hist, q1 - below, q2 - below, C, b1, c1, b2, c2);
        const int cnt = c2 + (int)hist[b2] - c1;
        if (tid == 0) C.g_n = 0;
        __syncthreads();
        if (cnt <= FB_CAP) {
            for (int i = tid; i < L; i += NT) {
                const float a = f(i);
                if (a >= lo && a <= hi) {
                    const int b = bucket(a, lo, scale);
                    if (b >= b1 && b <= b2) {
                        const int pos = atomicAdd(&C.g_n, 1);
                        if (pos < FB_CAP) buf[pos] = a;
                    }
                }
            }
            __syncthreads();
            const int s1 = q1 - below - c1, s2 = q2 - below - c1;
            float o1 = 0.f, o2 = 0.f;
            for (int t = tid; t < cnt; t += NT) {
                o1 = o2 = __int_as_float(0x7FC00000);
                rank_pick(buf, cnt, t, s1, s2, o1, o2);
                if (!isnan(o1)) C.g_v1 = o1;
                if (!isnan(o2)) C.g_v2 = o2;
            }
            __syncthreads();
            v1 = C.g_v1;
            v2 = C.g_v2;
            __syncthreads();
            return;
        }
        float nlo = FLT_MAX, nhi = -FLT_MAX;
        for (int i = tid; i < L; i += NT) {
            const float a = f(i);
            if (a >= lo && a <= hi) {
                const int b = bucket(a, lo, scale);
                if (b >= b1 && b <= b2) {
                    nlo = fminf(nlo, a);
                    nhi = fmaxf(nhi, a);
                }
            }
        }
        nlo = warp_min(nlo);
        nhi = warp_max(nhi);
        if ((tid & 31) == 0) {
            C.fred[tid >> 5] = nlo;
            C.fred[NWARP + (tid >> 5)] = nhi;
        }
        __syncthreads();
        lo = C.fred[0];
        hi = C.fred[NWARP];
        for (int i = 1; i < NWARP; ++i) {
            lo = fminf(lo, C.fred[i]);
            hi = fmaxf(hi, C.fred[NWARP + i]);
        }
        below += c1;
        __syncthreads();
    }
    if (tid == 0) atomicOr(err, ERR_SELECT_ITER);
    v1 = v2 = __int_as_float(0x7FC00000);
}

__device__ __forceinline__ double depth_from(double num, double spread)
{
    if (spread == 0.0) return num == 0.0 ? 1.0 : 0.0;
    return 1.0 / (1.0 + num / spread);
}

// G: directions per CTA (compile time); DP4: d rounded up to 4 when <= 16 (the
// directions are then held in registers), 0 for any d.
template <int G, int DP4>
__global__ void __launch_bounds__(NT, (G >= 4 ? 1 : 2)) k_pdap2(const TaskDev* __restrict__ tasks, const SlotDev* __restrict__ slots,
                                                 const DsDev* __restrict__ dsets, const float* __restrict__ U,
                                                 const float* __restrict__ z32, ResDev* __restrict__ res, int* err)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ Ctl C;
    const TaskDev T = tasks[blockIdx.x];
    const SlotDev& S = slots[T.slot];
    const DsDev D = dsets[S.ds];
    const int n = (int)D.n, ldx = D.ldx, d = D.d, dp4 = DP4 ? DP4 : ((d + 3) & ~3);
    const bool ap = (S.kind == 2);
    const int tid = threadIdx.x;
    const int npad = (n + 3) & ~3;
    float* keys = sm;                                          // G x npad
    float* uS = keys + (size_t)G * npad;                       // G x ldx
    unsigned* hist = reinterpret_cast<unsigned*>(uS + (size_t)G * ldx);   // G x NB
    float* buf = reinterpret_cast<float*>(hist + (size_t)G * NB);        // G x 2 x CAP

    const int GA = T.nj;   // live directions; slots GA..G-1 are inert
    for (int e = tid; e < G * ldx; e += NT) uS[e] = (e / ldx < GA) ? U[S.uoff + (int64_t)T.j0 * ldx + e] : 0.0f;
    for (int e = tid; e < G * NB; e += NT) hist[e] = 0u;
    if (tid < MAXG * 2) {
        const float qnan = __int_as_float(0x7FC00000);
        C.v1[tid >> 1][tid & 1] = qnan;
        C.v2[tid >> 1][tid & 1] = qnan;
    }
    if (tid < MAXG) {
        C.npos[tid] = 0;
        C.fb[tid] = tid < GA ? 0 : 3;
    }
    __syncthreads();
    // per-direction bucket range: the centre's projection +- 5 sigma_u (sigma_u^2 = u' Cov u),
    // or +- the radius about the centre when no covariance is kept.  Keys outside the range go
    // to the edge buckets, which keeps the bucket map monotone.
    if (tid < G) {
        const int g = tid;
        const float* u = uS + g * ldx;
        float a = 0.0f, yc = 0.0f;
        const float* zr = z32 + S.zoff32;
        for (int l = 0; l < dp4; ++l) a = fmaf(u[l], zr[l], a);   // y_z: same arithmetic as the keys
        for (int l = 0; l < d; ++l) yc = fmaf(u[l], D.center[l], yc);
        float half = D.rc * 1.0001f;
        if (D.cov) {
            float q = 0.0f;
            for (int r = 0; r < d; ++r) {
                float t = 0.0f;
                for (int c2 = 0; c2 < d; ++c2) t = fmaf(D.cov[r * d + c2], u[c2], t);
                q = fmaf(u[r], t, q);
            }
            const float sg = sqrtf(fmaxf(q, 0.0f));
            if (sg > 0.0f && 5.0f * sg < half) half = 5.0f * sg;
            C.scale[g] = sg;   // kept for the deviation range
        } else {
            C.scale[g] = half;
        }
        if (!(half > 0.0f)) half = fmaxf(fabsf(yc), 1.0f);
        C.yz[g] = a;
        C.lo_b[g] = yc - half;
        C.sc_y[g] = __fdiv_rn((float)NB, __fadd_rn(half, half));
        C.off_y[g] = __fmul_rn(-C.lo_b[g], C.sc_y[g]);
    }
    __syncthreads();

    // ---- pass A: keys + bucket counts ----------------------------------------------
    {
        float of[G], sc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            of[g] = C.off_y[g];
            sc[g] = C.sc_y[g];
        }
        auto emit = [&](int i, const float (&acc)[G]) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                keys[(size_t)g * npad + i] = acc[g];
                atomicAdd(&hist[g * NB + bucket_fma(acc[g], sc[g], of[g])], 1u);
            }
        };
        if (DP4 > 0) {
            float4 ur[G][DP4 > 0 ? DP4 / 4 : 1];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int c = 0; c < DP4 / 4; ++c) ur[g][c] = *reinterpret_cast<const float4*>(uS + g * ldx + 4 * c);
            // two points per iteration: both rows' loads are in flight together
            for (int i = tid; i < n; i += 2 * NT) {
                const int i2 = i + NT;
                const bool two = i2 < n;
                const float4* xa = reinterpret_cast<const float4*>(D.X32 + (int64_t)i * ldx);
                const float4* xb = reinterpret_cast<const float4*>(D.X32 + (int64_t)(two ? i2 : i) * ldx);
                float4 va[DP4 > 0 ? DP4 / 4 : 1], vb[DP4 > 0 ? DP4 / 4 : 1];
#pragma unroll
                for (int c = 0; c < DP4 / 4; ++c) {
                    va[c] = xa[c];
                    vb[c] = xb[c];
                }
                float acc[G], acc2[G];
#pragma unroll
                for (int g = 0; g < G; ++g) acc[g] = acc2[g] = 0.f;
#pragma unroll
                for (int c = 0; c < DP4 / 4; ++c) {
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        acc[g] = fmaf(ur[g][c].x, va[c].x, acc[g]);
                        acc[g] = fmaf(ur[g][c].y, va[c].y, acc[g]);
                        acc[g] = fmaf(ur[g][c].z, va[c].z, acc[g]);
                        acc[g] = fmaf(ur[g][c].w, va[c].w, acc[g]);
                        acc2[g] = fmaf(ur[g][c].x, vb[c].x, acc2[g]);
                        acc2[g] = fmaf(ur[g][c].y, vb[c].y, acc2[g]);
                        acc2[g] = fmaf(ur[g][c].z, vb[c].z, acc2[g]);
                        acc2[g] = fmaf(ur[g][c].w, vb[c].w, acc2[g]);
                    }
                }
                emit(i, acc);
                if (two) emit(i2, acc2);
            }
        } else {
            for (int i = tid; i < n; i += NT) {
                const float4* xr = reinterpret_cast<const float4*>(D.X32 + (int64_t)i * ldx);
                float acc[G];
#pragma unroll
                for (int g = 0; g < G; ++g) acc[g] = 0.f;
                for (int l = 0; l < dp4; l += 4) {
                    const float4 x = xr[l >> 2];
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const float4 u = *reinterpret_cast<const float4*>(uS + g * ldx + l);
                        acc[g] = fmaf(u.x, x.x, acc[g]);
                        acc[g] = fmaf(u.y, x.y, acc[g]);
                        acc[g] = fmaf(u.z, x.z, acc[g]);
                        acc[g] = fmaf(u.w, x.w, acc[g]);
                    }
                }
                emit(i, acc);
            }
        }
    }
    __syncthreads();

    const int k1 = (n - 1) / 2, k2 = n / 2;
    const int npos_guess = (n & 1) ? (n - 1) / 2 : n / 2;
    // ---- bucket runs of the wanted ranks ----------------------------------------
    for (int g = 0; g < GA; ++g) {
        int ba, ca, bb, cb;
        find_buckets(hist + g * NB, k1, k2, C, ba, ca, bb, cb);
        if (tid == 0) {
            C.b_lo[g][0] = ba;
            C.b_hi[g][0] = bb;
            C.c_lo[g][0] = ca;
            C.cnt[g][0] = cb + (int)hist[g * NB + bb] - ca;
            C.fill[g][0] = 0;
            C.fb[g] = C.cnt[g][0] > CAP ? 1 : 0;
        }
        if (ap) {
            const int base = n - npos_guess;
            const int r3 = base + (npos_guess - 1) / 2, r4 = base + npos_guess / 2;
            if (npos_guess > 0) {
                find_buckets(hist + g * NB, r3, r4, C, ba, ca, bb, cb);
                if (tid == 0) {
                    C.b_lo[g][1] = ba;
                    C.b_hi[g][1] = bb;
                    C.c_lo[g][1] = ca;
                    C.cnt[g][1] = cb + (int)hist[g * NB + bb] - ca;
                    if (C.cnt[g][1] > CAP) C.fb[g] = 1;
                }
            } else if (tid == 0) {
                C.b_lo[g][1] = 1;
                C.b_hi[g][1] = 0;   // empty run
                C.c_lo[g][1] = 0;
                C.cnt[g][1] = 0;
            }
            if (tid == 0) C.fill[g][1] = 0;
        }
        __syncthreads();
    }

    // ---- pass C: gather the runs ------------------------------------------------
    {
        int bl0[G], bw0[G], bl1[G], bw1[G];
        float of[G], sc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            // a run that is off gets a start no bucket index can reach: (b - start) is then
            // never <= 0 as an unsigned number
            const bool on = !C.fb[g];
            of[g] = C.off_y[g];
            sc[g] = C.sc_y[g];
            bl0[g] = on ? C.b_lo[g][0] : (1 << 30);
            bw0[g] = on ? C.b_hi[g][0] - C.b_lo[g][0] : 0;
            bl1[g] = (ap && on) ? C.b_lo[g][1] : (1 << 30);
            bw1[g] = (ap && on) ? C.b_hi[g][1] - C.b_lo[g][1] : 0;
        }
        auto gather = [&](int g, float y) {
            const int b = bucket_fma(y, sc[g], of[g]);
            if ((unsigned)(b - bl0[g]) <= (unsigned)bw0[g]) {
                const int pos = atomicAdd(&C.fill[g][0], 1);
                if (pos < CAP) buf[(g * 2 + 0) * CAP + pos] = y;
            }
            if (ap && (unsigned)(b - bl1[g]) <= (unsigned)bw1[g]) {
                const int pos = atomicAdd(&C.fill[g][1], 1);
                if (pos < CAP) buf[(g * 2 + 1) * CAP + pos] = y;
            }
        };
        const int n4 = n & ~3;
        for (int i = 4 * tid; i < n4; i += 4 * NT) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const float4 y4 = *reinterpret_cast<const float4*>(keys + (size_t)g * npad + i);
                gather(g, y4.x);
                gather(g, y4.y);
                gather(g, y4.z);
                gather(g, y4.w);
            }
        }
        for (int i = n4 + tid; i < n; i += NT) {
#pragma unroll
            for (int g = 0; g < G; ++g) gather(g, keys[(size_t)g * npad + i]);
        }
    }
    __syncthreads();

    // ---- exact ranks within the gathered keys -------------------------------------
    for (int g = 0; g < G; ++g) {
        if (C.fb[g]) continue;
        const int cnt = C.cnt[g][0];
        const int s1 = k1 - C.c_lo[g][0], s2 = k2 - C.c_lo[g][0];
        for (int t = tid; t < cnt; t += NT) {
            float o1 = __int_as_float(0x7FC00000), o2 = o1;
            rank_pick(buf + (g * 2) * CAP, cnt, t, s1, s2, o1, o2);
            if (!isnan(o1)) C.v1[g][0] = o1;
            if (!isnan(o2)) C.v2[g][0] = o2;
        }
    }
    if (tid < MAXG) C.nle[tid] = 0;
    __syncthreads();
    if (ap) {
        // #(y <= med) = #(y <= m1): keys below the run plus gathered keys <= m1
        for (int g = 0; g < G; ++g) {
            if (C.fb[g]) continue;
            const float m1 = C.v1[g][0];
            int c = 0;
            for (int t = tid; t < C.cnt[g][0]; t += NT) c += (buf[(g * 2) * CAP + t] <= m1);
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
            if ((tid & 31) == 0 && c) atomicAdd(&C.nle[g], c);
        }
        __syncthreads();
        for (int g = 0; g < G; ++g) {
            if (C.fb[g]) continue;
            const int nle = C.c_lo[g][0] + C.nle[g];
            const int npos = n - nle;
            if (tid == 0) C.npos[g] = npos;
            if (npos == 0) continue;
            const int base = n - npos;
            const int r3 = base + (npos - 1) / 2, r4 = base + npos / 2;
            const int s3 = r3 - C.c_lo[g][1], s4 = r4 - C.c_lo[g][1];
            const int cnt = C.cnt[g][1];
            if (s3 < 0 || s4 >= cnt) {
                if (tid == 0) C.fb[g] = 2;   // the positive count differed from the guess
                continue;
            }
            for (int t = tid; t < cnt; t += NT) {
                float o1 = __int_as_float(0x7FC00000), o2 = o1;
                rank_pick(buf + (g * 2 + 1) * CAP, cnt, t, s3, s4, o1, o2);
                if (!isnan(o1)) C.v1[g][1] = o1;
                if (!isnan(o2)) C.v2[g][1] = o2;
            }
        }
        __syncthreads();
    } else {
        // ---- D_P: |y - med| histogram over [0, 4 sigma_u] (edge bucket clamps), gather, ranks
        for (int e = tid; e < G * NB; e += NT) hist[e] = 0u;
        if (tid < G) {
            const float m = __fmul_rn(__fadd_rn(C.v1[tid][0], C.v2[tid][0]), 0.5f);
            float dmax = D.cov ? 4.0f * C.scale[tid] : 0.0f;
            const float hard = __fmul_rn(__fadd_rn(D.rc, fabsf(m - C.lo_b[tid] - 0.5f * (float)NB / C.sc_y[tid])),
                                         1.0001f);
            if (!(dmax > 0.0f) || dmax > hard) dmax = hard;
            if (!(dmax > 0.0f)) dmax = 1.0f;
            C.cen[tid] = m;
            C.sc_d[tid] = __fdiv_rn((float)NB, dmax);
        }
        __syncthreads();
        {
            float cen[G], scl[G];
            bool on[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                on[g] = !C.fb[g];
                cen[g] = C.cen[g];
                scl[g] = C.sc_d[g];
            }
            auto add = [&](int g, float y) {
                const float dv = fabsf(__fsub_rn(y, cen[g]));
                atomicAdd(&hist[g * NB + bucket_fma(dv, scl[g], 0.0f)], 1u);
            };
            const int n4 = n & ~3;
            for (int i = 4 * tid; i < n4; i += 4 * NT) {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (on[g]) {
                        const float4 y4 = *reinterpret_cast<const float4*>(keys + (size_t)g * npad + i);
                        add(g, y4.x);
                        add(g, y4.y);
                        add(g, y4.z);
                        add(g, y4.w);
                    }
                }
            }
            for (int i = n4 + tid; i < n; i += NT) {
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (on[g]) add(g, keys[(size_t)g * npad + i]);
            }
        }
        __syncthreads();
        for (int g = 0; g < G; ++g) {
            if (C.fb[g]) continue;
            int ba, ca, bb, cb;
            find_buckets(hist + g * NB, k1, k2, C, ba, ca, bb, cb);
            if (tid == 0) {
                C.b_lo[g][1] = ba;
                C.b_hi[g][1] = bb;
                C.c_lo[g][1] = ca;
                C.cnt[g][1] = cb + (int)hist[g * NB + bb] - ca;
                C.fill[g][1] = 0;
                if (C.cnt[g][1] > CAP) C.fb[g] = 2;
            }
            __syncthreads();
        }
        {
            float cen[G], scl[G];
            int bl[G], bw[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                cen[g] = C.cen[g];
                scl[g] = C.sc_d[g];
                bl[g] = !C.fb[g] ? C.b_lo[g][1] : (1 << 30);
                bw[g] = !C.fb[g] ? C.b_hi[g][1] - C.b_lo[g][1] : 0;
            }
            auto gather = [&](int g, float y) {
                const float dv = fabsf(__fsub_rn(y, cen[g]));
                const int b = bucket_fma(dv, scl[g], 0.0f);
                if ((unsigned)(b - bl[g]) <= (unsigned)bw[g]) {
                    const int pos = atomicAdd(&C.fill[g][1], 1);
                    if (pos < CAP) buf[(g * 2 + 1) * CAP + pos] = dv;
                }
            };
            const int n4 = n & ~3;
            for (int i = 4 * tid; i < n4; i += 4 * NT) {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const float4 y4 = *reinterpret_cast<const float4*>(keys + (size_t)g * npad + i);
                    gather(g, y4.x);
                    gather(g, y4.y);
                    gather(g, y4.z);
                    gather(g, y4.w);
                }
            }
            for (int i = n4 + tid; i < n; i += NT) {
#pragma unroll
                for (int g = 0; g < G; ++g) gather(g, keys[(size_t)g * npad + i]);
            }
        }
        __syncthreads();
        for (int g = 0; g < G; ++g) {
            if (C.fb[g]) continue;
            const int cnt = C.cnt[g][1];
            const int s1 = k1 - C.c_lo[g][1], s2 = k2 - C.c_lo[g][1];
            for (int t = tid; t < cnt; t += NT) {
                float o1 = __int_as_float(0x7FC00000), o2 = o1;
                rank_pick(buf + (g * 2 + 1) * CAP, cnt, t, s1, s2, o1, o2);
                if (!isnan(o1)) C.v1[g][1] = o1;
                if (!isnan(o2)) C.v2[g][1] = o2;
            }
        }
        __syncthreads();
    }

    // ---- fallback directions: iterated bucket selection over their keys ---------
    for (int g = 0; g < G; ++g) {
        const int fb = C.fb[g];
        if (fb == 0 || fb == 3) continue;
        const float* y = keys + (size_t)g * npad;
        // exact range of this direction's keys
        float kl = FLT_MAX, kh = -FLT_MAX;
        for (int i = tid; i < n; i += NT) {
            kl = fminf(kl, y[i]);
            kh = fmaxf(kh, y[i]);
        }
        kl = warp_min(kl);
        kh = warp_max(kh);
        __syncthreads();
        if ((tid & 31) == 0) {
            C.fred[tid >> 5] = kl;
            C.fred[NWARP + (tid >> 5)] = kh;
        }
        __syncthreads();
        kl = C.fred[0];
        kh = C.fred[NWARP];
        for (int i = 1; i < NWARP; ++i) {
            kl = fminf(kl, C.fred[i]);
            kh = fmaxf(kh, C.fred[NWARP + i]);
        }
        __syncthreads();
        float m1, m2;
        if (fb == 1) {
            select_generic([&](int i) { return y[i]; }, n, k1, k2, kl, kh, hist, buf, C, m1, m2, err);
            if (tid == 0) {
                C.v1[g][0] = m1;
                C.v2[g][0] = m2;
            }
            __syncthreads();
        } else {
            m1 = C.v1[g][0];
            m2 = C.v2[g][0];
        }
        if (ap) {
            int c = 0;
            for (int i = tid; i < n; i += NT) c += (y[i] <= m1);
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
            __syncthreads();
            if ((tid & 31) == 0) C.red[tid >> 5] = c;
            __syncthreads();
            int nle = 0;
            for (int i = 0; i < NWARP; ++i) nle += C.red[i];
            const int npos = n - nle;
            if (tid == 0) C.npos[g] = npos;
            float p1 = m1, p2 = m1;
            if (npos > 0)
                select_generic([&](int i) { return y[i]; }, n, nle + (npos - 1) / 2, nle + npos / 2, kl, kh, hist,
                               buf, C, p1, p2, err);
            if (tid == 0) {
                C.v1[g][1] = p1;
                C.v2[g][1] = p2;
            }
        } else {
            const float m = __fmul_rn(__fadd_rn(m1, m2), 0.5f);
            const float dmax = fmaxf(fabsf(__fsub_rn(kl, m)), fabsf(__fsub_rn(kh, m)));
            float a1, a2;
            select_generic([&](int i) { return fabsf(__fsub_rn(y[i], m)); }, n, k1, k2, 0.0f, dmax, hist, buf, C, a1,
                           a2, err);
            if (tid == 0) {
                C.v1[g][1] = a1;
                C.v2[g][1] = a2;
            }
        }
        __syncthreads();
    }

    // ---- depths (FP64 on a handful of values) --------------------------------------
    if (tid < GA) {
        const int g = tid;
        const double med = ((double)C.v1[g][0] + (double)C.v2[g][0]) * 0.5;
        const double yzv = (double)C.yz[g];
        double depth;
        if (ap) {
            const double madp =
                C.npos[g] > 0 ? (((double)C.v1[g][1] - med) + ((double)C.v2[g][1] - med)) * 0.5 : 0.0;
            depth = depth_from(yzv - med > 0.0 ? yzv - med : 0.0, madp);
        } else {
            const double mad = ((double)C.v1[g][1] + (double)C.v2[g][1]) * 0.5;
            depth = depth_from(fabs(yzv - med), mad);
        }
        res[S.roff + T.j0 + g] = ResDev{depth, -1};
    }
}

}  // namespace

size_t pdap_smem_bytes(int n, int group, int ldx)
{
    const size_t npad = ((size_t)n + 3) & ~(size_t)3;
    return sizeof(float) * ((size_t)group * npad + (size_t)group * ldx) + sizeof(unsigned) * (size_t)group * NB +
           sizeof(float) * (size_t)group * 2 * CAP;
}

size_t pdap_smem_limit()
{
    // opt-in maximum per CTA (227 KB) minus the kernel's static control block
    return 232448 - sizeof(Ctl) - 256;
}

int pdap_max_group(int n, int ldx, int m)
{
    // G in {1, 2, 4}: the largest that fits two CTAs per SM when that is at least 2, else the
    // largest that fits one CTA per SM
    const size_t one = pdap_smem_limit(), two = 110 * 1024;
    int g_one = 0, g_two = 0;
    for (int g = 1; g <= MAXG && g <= m; g *= 2) {
        if (pdap_smem_bytes(n, g, ldx) <= one) g_one = g;
        if (pdap_smem_bytes(n, g, ldx) <= two) g_two = g;
    }
    if (g_two >= 2) return g_two;
    return g_one;
}

template <int G, int DP4>
static cudaError_t launch_t(const TaskDev* tasks, int ntasks, size_t smem, const SlotDev* slots, const DsDev* ds,
                            const float* U, const float* z32, ResDev* res, int* err, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(k_pdap2<G, DP4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();   // do not leave the failure pending for an unrelated later call
        return e;
    }
    k_pdap2<G, DP4><<<ntasks, NT, smem, st>>>(tasks, slots, ds, U, z32, res, err);
    return cudaGetLastError();
}

template <int G>
static cudaError_t launch_g(int dp4, const TaskDev* tasks, int ntasks, size_t smem, const SlotDev* slots,
                            const DsDev* ds, const float* U, const float* z32, ResDev* res, int* err, cudaStream_t st)
{
    switch (dp4) {
    case 4: return launch_t<G, 4>(tasks, ntasks, smem, slots, ds, U, z32, res, err, st);
    case 8: return launch_t<G, 8>(tasks, ntasks, smem, slots, ds, U, z32, res, err, st);
    case 12: return launch_t<G, 12>(tasks, ntasks, smem, slots, ds, U, z32, res, err, st);
    case 16: return launch_t<G, 16>(tasks, ntasks, smem, slots, ds, U, z32, res, err, st);
    default: return launch_t<G, 0>(tasks, ntasks, smem, slots, ds, U, z32, res, err, st);
    }
}

int pdap_dp4_class(int d)
{
    const int dp4 = (d + 3) & ~3;
    return dp4 <= 16 ? dp4 : 0;
}

cudaError_t launch_pdap(const TaskDev* tasks, int ntasks, size_t smem, int group, int dp4, const SlotDev* slots,
                        const DsDev* ds, const float* U, const float* z32, ResDev* res, int* err, cudaStream_t st)
{
    if (ntasks <= 0) return cudaSuccess;
    if (smem > pdap_smem_limit()) return cudaErrorInvalidValue;
    switch (group) {
    case 1: return launch_g<1>(dp4, tasks, ntasks, smem, slots, ds, U, z32, res, err, st);
    case 2: return launch_g<2>(dp4, tasks, ntasks, smem, slots, ds, U, z32, res, err, st);
    case 4: return launch_g<4>(dp4, tasks, ntasks, smem, slots, ds, U, z32, res, err, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rrs
