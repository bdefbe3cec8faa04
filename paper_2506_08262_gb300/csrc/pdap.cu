// Projection depth D_P and asymmetric projection depth D_AP (Sec. 2) for a block
// of directions: y_i = u'x_i in FP32, exact order statistics (median, MAD,
// MAD_+) of the FP32 keys, depth in FP64 from those few values.
//
// One CTA handles G <= 4 directions of one query with the G*n keys resident in
// shared memory, or, when n is beyond what shared memory holds, G = 2
// directions whose keys stay outside: formed once by a keys kernel and read
// from global memory at every pass, or (allocation-free entry point)
// recomputed from X at every pass; the arithmetic is the same throughout, and
// so are the values.  The whole CTA projects (pass A: every point on the G
// directions, keys stored, each added to a 2048-bucket histogram over
// u'c +- 5 sigma_u, bucket = monotone FP32 map of the key).  Then the CTA
// splits into G groups of (CTA threads)/G, one per direction, each synchronising
// on its own named barrier, so the directions never wait for one another:
//   median  find the buckets of the median ranks, gather their keys (and, for
//           D_AP, the keys of the buckets expected to hold the MAD_+ ranks),
//           rank them exactly;
//   D_P     histogram of |y - med|, gather the MAD buckets, rank (MAD).
// Bucket maps are monotone, so every bucket holds a contiguous run of ranks
// and the gathered keys contain the wanted order statistics.  When a run holds
// more keys than the gather buffer, or the D_AP guess of the positive count
// was wrong, the group falls back to an iterated bucket selection over its
// keys.  No per-element work uses FP64.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "rrs_internal.h"

namespace rrs {
namespace {

constexpr int NT = 512;              // threads per CTA for G = 1, 2 (two CTAs per SM)
constexpr int NT4 = 1024;            // threads per CTA for G = 4 (one CTA per SM)
constexpr int NWARP = NT4 / 32;      // largest warp count of a CTA
template <int G>
__host__ __device__ constexpr int cta_threads()
{
    return G == 4 ? NT4 : NT;
}
constexpr int NB = 2048;     // buckets per direction
constexpr int CAP = 256;     // gathered keys per direction and target
constexpr int MAXG = 4;
constexpr int FB_NB = NB;    // fallback histogram (reuses the bucket area)
constexpr int FB_CAP = 2 * CAP;  // fallback gather buffer: a direction's two gather areas

// Per-direction constants and per-group scratch: after the projection pass,
// group g (CTA threads / G) works on direction g alone and synchronises with
// the named barrier 1 + g, so the directions of a CTA never wait for each other.
struct Ctl {
    float lo_b[MAXG], sc_y[MAXG];      // bucket map of the keys: about (y - lo_b) * sc_y
    float off_y[MAXG];                 // -lo_b * sc_y (bucket_fma offset)
    float scale[MAXG];                 // sigma_u (or the radius) of each direction
    int red[MAXG][NWARP];
    float fred[MAXG][2 * NWARP];
    int fill[MAXG][2];
    int f_b1[MAXG], f_c1[MAXG], f_b2[MAXG], f_c2[MAXG];   // bucket search results
    float pv1[MAXG], pv2[MAXG];                           // rank pick results
    int pi1[MAXG], pi2[MAXG];                             // their point indices
    int gn[MAXG];
    int gi[MAXG];                                         // smallest index of a tied run (fallback)
    double y64[MAXG][4];                                  // FP64 projections of the selected points
};

template <int GS>
struct Grp {
    int g, t;   // direction (group) index, thread index within the group
    __device__ __forceinline__ void sync() const
    {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(GS) : "memory");
    }
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

// Group sum of one int per thread (every thread gets the total).
template <int GS>
__device__ int gsum(const Grp<GS>& q, int c, Ctl& C)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if ((q.t & 31) == 0) C.red[q.g][q.t >> 5] = c;
    q.sync();
    int s = 0;
#pragma unroll
    for (int i = 0; i < GS / 32; ++i) s += C.red[q.g][i];
    q.sync();
    return s;
}

// Group min and max.
template <int GS>
__device__ void gminmax(const Grp<GS>& q, float lo, float hi, Ctl& C, float& olo, float& ohi)
{
    lo = warp_min(lo);
    hi = warp_max(hi);
    if ((q.t & 31) == 0) {
        C.fred[q.g][q.t >> 5] = lo;
        C.fred[q.g][NWARP + (q.t >> 5)] = hi;
    }
    q.sync();
    olo = C.fred[q.g][0];
    ohi = C.fred[q.g][NWARP];
#pragma unroll
    for (int i = 1; i < GS / 32; ++i) {
        olo = fminf(olo, C.fred[q.g][i]);
        ohi = fmaxf(ohi, C.fred[q.g][NWARP + i]);
    }
    q.sync();
}

// Exclusive scan of h[0..NB) by the group; the bucket holding rank ra and the
// one holding rank rb (ra <= rb, both below the total), with the keys below each.
template <int GS>
__device__ void gfind(const Grp<GS>& q, const unsigned* h, int ra, int rb, Ctl& C, int& ba, int& ca, int& bb, int& cb)
{
    constexpr int PER = NB / GS;   // 4, 8 or 16 consecutive buckets per thread, read as uint4
    const int lane = q.t & 31, w = q.t >> 5;
    int own = 0;
    unsigned v[PER];
    const uint4* h4 = reinterpret_cast<const uint4*>(h + q.t * PER);
#pragma unroll
    for (int k = 0; k < PER / 4; ++k) {
        const uint4 a = h4[k];
        v[4 * k] = a.x;
        v[4 * k + 1] = a.y;
        v[4 * k + 2] = a.z;
        v[4 * k + 3] = a.w;
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) own += (int)v[k];
    int incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) C.red[q.g][w] = incl;
    q.sync();
    int base = 0;
    for (int i = 0; i < w; ++i) base += C.red[q.g][i];
    int c = base + incl - own;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int hk = (int)v[k];
        if (hk > 0) {
            if (c <= ra && ra < c + hk) {
                C.f_b1[q.g] = q.t * PER + k;
                C.f_c1[q.g] = c;
            }
            if (c <= rb && rb < c + hk) {
                C.f_b2[q.g] = q.t * PER + k;
                C.f_c2[q.g] = c;
            }
        }
        c += hk;
    }
    q.sync();
    ba = C.f_b1[q.g];
    ca = C.f_c1[q.g];
    bb = C.f_b2[q.g];
    cb = C.f_c2[q.g];
    q.sync();
}

// Values and point indices of the 0-based ranks s1 <= s2 among the pairs (buf, ib)[0..cnt), ordered by
// value and then by point index, by the group.  The indices of one buffer are distinct, so every rank
// names one pair and the choice among equal values never depends on the gather order.
template <int GS>
__device__ void gpick(const Grp<GS>& q, const float* buf, const int* ib, int cnt, int s1, int s2, Ctl& C, float& o1,
                      float& o2, int& i1, int& i2)
{
    for (int t = q.t; t < cnt; t += GS) {
        const float v = buf[t];
        const int iv = ib[t];
        int r = 0;
        for (int s = 0; s < cnt; ++s) {
            const float w2 = buf[s];
            r += (w2 < v) | ((w2 == v) & (ib[s] < iv));
        }
        if (r == s1) {
            C.pv1[q.g] = v;
            C.pi1[q.g] = iv;
        }
        if (r == s2) {
            C.pv2[q.g] = v;
            C.pi2[q.g] = iv;
        }
    }
    q.sync();
    o1 = C.pv1[q.g];
    o2 = C.pv2[q.g];
    i1 = C.pi1[q.g];
    i2 = C.pi2[q.g];
    q.sync();
}

// Inclusive prefix sums of h[0..NB) in place, by the group.
template <int GS>
__device__ void gprefix(const Grp<GS>& q, unsigned* h, Ctl& C)
{
    constexpr int PER = NB / GS;
    const int lane = q.t & 31, w = q.t >> 5;
    unsigned v[PER];
    uint4* h4 = reinterpret_cast<uint4*>(h + q.t * PER);
#pragma unroll
    for (int k = 0; k < PER / 4; ++k) {
        const uint4 a = h4[k];
        v[4 * k] = a.x;
        v[4 * k + 1] = a.y;
        v[4 * k + 2] = a.z;
        v[4 * k + 3] = a.w;
    }
#pragma unroll
    for (int k = 1; k < PER; ++k) v[k] += v[k - 1];
    int incl = (int)v[PER - 1];
    const int own = incl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) C.red[q.g][w] = incl;
    q.sync();
    int base = incl - own;
    for (int i = 0; i < w; ++i) base += C.red[q.g][i];
#pragma unroll
    for (int k = 0; k < PER / 4; ++k)
        h4[k] = make_uint4(v[4 * k] + base, v[4 * k + 1] + base, v[4 * k + 2] + base, v[4 * k + 3] + base);
    q.sync();
}

// Generic exact selection of ranks q1 <= q2 over one direction's values f(0..L-1),
// all in [lo, hi], by iterated bucketing (the fallback path); hist, buf and ibuf are the
// direction's own areas.  Returns the values and the point indices of the two ranks.
template <int GS, class F>
__device__ void gselect(const Grp<GS>& q, F f, int L, int q1, int q2, float lo, float hi, unsigned* hist, float* buf,
                        int* ibuf, Ctl& C, float& v1, float& v2, int& i1, int& i2, int* err)
{
    int below = 0;
    for (int iter = 0; iter < 24; ++iter) {
        if (!(lo < hi)) {
            // every remaining candidate equals lo: both ranks hold that value, taken at the
            // smallest point index that holds it
            if (q.t == 0) C.gi[q.g] = 0x7FFFFFFF;
            q.sync();
            for (int i = q.t; i < L; i += GS) {
                if (f(i) == lo) {
                    atomicMin(&C.gi[q.g], i);
                    break;
                }
            }
            q.sync();
            v1 = v2 = lo;
            i1 = i2 = C.gi[q.g];
            q.sync();
            return;
        }
        float scale = __fdiv_rn((float)FB_NB, __fsub_rn(hi, lo));
        if (!(scale <= FLT_MAX)) scale = FLT_MAX;
        for (int b = q.t; b < FB_NB / 4; b += GS) reinterpret_cast<uint4*>(hist)[b] = make_uint4(0u, 0u, 0u, 0u);
        q.sync();
        for (int i = q.t; i < L; i += GS) {
            const float a = f(i);
            if (a >= lo && a <= hi) atomicAdd(&hist[bucket(a, lo, scale)], 1u);
        }
        q.sync();
        int b1, c1, b2, c2;
        gfind(q, hist, q1 - below, q2 - below, C, b1, c1, b2, c2);
        const int cnt = c2 + (int)hist[b2] - c1;
        if (q.t == 0) C.gn[q.g] = 0;
        q.sync();
        if (cnt <= FB_CAP) {
            for (int i = q.t; i < L; i += GS) {
                const float a = f(i);
                if (a >= lo && a <= hi) {
                    const int b = bucket(a, lo, scale);
                    if (b >= b1 && b <= b2) {
                        const int pos = atomicAdd(&C.gn[q.g], 1);
                        if (pos < FB_CAP) {
                            buf[pos] = a;
                            ibuf[pos] = i;
                        }
                    }
                }
            }
            q.sync();
            gpick(q, buf, ibuf, cnt, q1 - below - c1, q2 - below - c1, C, v1, v2, i1, i2);
            return;
        }
        float nlo = FLT_MAX, nhi = -FLT_MAX;
        for (int i = q.t; i < L; i += GS) {
            const float a = f(i);
            if (a >= lo && a <= hi) {
                const int b = bucket(a, lo, scale);
                if (b >= b1 && b <= b2) {
                    nlo = fminf(nlo, a);
                    nhi = fmaxf(nhi, a);
                }
            }
        }
        gminmax(q, nlo, nhi, C, lo, hi);
        below += c1;
    }
    if (q.t == 0) atomicOr(err, ERR_SELECT_ITER);
    v1 = v2 = __int_as_float(0x7FC00000);
    i1 = i2 = -1;
}

// 1 / (1 + num / spread) = spread / (spread + num) for num, spread >= 0 (FP64 inputs, exact differences
// of FP32 order statistics).  GB300 issues FP64 at a fraction of the FP32 rate, so the one division is
// done in FP32 (relative error a few 2^-24) whenever both operands and the quotient are safely normal
// FP32 numbers, and in FP64 otherwise.
__device__ __forceinline__ double depth_from(double num, double spread)
{
    if (spread == 0.0) return num == 0.0 ? 1.0 : 0.0;
    const double den = spread + num;
    if (spread >= 1e-30 && den <= 1e30 && spread >= 1e-20 * den)
        return (double)__fdiv_rn((float)spread, (float)den);
    return spread / den;
}

// Key u'x for d <= 16 (DP4 = d rounded up to 4): two sequential FMA chains over the two
// halves of the DP4 dims, added (two independent chains per key).  Keys and y_z are formed
// the same way whatever the group size, so results never depend on it.
template <int DP4>
__device__ __forceinline__ float key_halves(const float* u, const float* x)
{
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int l = 0; l < DP4 / 2; ++l) p0 = fmaf(u[l], x[l], p0);
#pragma unroll
    for (int l = DP4 / 2; l < DP4; ++l) p1 = fmaf(u[l], x[l], p1);
    return __fadd_rn(p0, p1);
}

// One direction's keys held in an array: shared memory (resident keys) or device memory (keys formed
// by launch_pdap_keys when they do not fit shared memory).
struct KeysArray {
    const float* y;
    __device__ __forceinline__ float get(int i) const { return y[i]; }
    __device__ __forceinline__ float4 get4(int i) const { return *reinterpret_cast<const float4*>(y + i); }
};

// One direction's keys recomputed from the FP32 rows of X with the projection pass's arithmetic
// (two half chains for d <= 16, one sequential FMA chain otherwise), so every pass sees the values
// a resident key would hold.  u: the direction in shared memory, dp4 floats (zero padded).
template <int DP4>
struct KeysRecomputed {
    const float* X;
    const float* u;
    int ldx, dp4;
    __device__ __forceinline__ float get(int i) const
    {
        const float4* xr = reinterpret_cast<const float4*>(X + (int64_t)i * ldx);
        if (DP4 > 0) {
            constexpr int D4 = DP4 > 0 ? DP4 : 4;
            float xv[D4], uv[D4];
#pragma unroll
            for (int c = 0; c < D4 / 4; ++c) {
                const float4 t4 = xr[c];
                const float4 u4 = *reinterpret_cast<const float4*>(u + 4 * c);
                xv[4 * c] = t4.x;
                xv[4 * c + 1] = t4.y;
                xv[4 * c + 2] = t4.z;
                xv[4 * c + 3] = t4.w;
                uv[4 * c] = u4.x;
                uv[4 * c + 1] = u4.y;
                uv[4 * c + 2] = u4.z;
                uv[4 * c + 3] = u4.w;
            }
            return key_halves<D4>(uv, xv);
        }
        float acc = 0.f;
        for (int l = 0; l < dp4; l += 4) {
            const float4 x = xr[l >> 2];
            const float4 w = *reinterpret_cast<const float4*>(u + l);
            acc = fmaf(w.x, x.x, acc);
            acc = fmaf(w.y, x.y, acc);
            acc = fmaf(w.z, x.z, acc);
            acc = fmaf(w.w, x.w, acc);
        }
        return acc;
    }
    __device__ __forceinline__ float4 get4(int i) const { return make_float4(get(i), get(i + 1), get(i + 2), get(i + 3)); }
};

// FP64 projection u'x_i of point i: one sequential FMA chain over the dims, from the FP64 rows when
// the data came in FP64 (the direction generator forms the query's y_z = u'z the same way, so a query
// equal to a data point projects to the same value).  Every product of an FP32 direction component and
// an FP32 (or FP64) coordinate is rounded at most once per added term.
__device__ __forceinline__ double proj64(const DsDev& D, const float* u, int i)
{
    double acc = 0.0;
    if (D.X64) {
        const double* xr = D.X64 + (int64_t)i * D.d;
        for (int l = 0; l < D.d; ++l) acc = __fma_rn((double)u[l], xr[l], acc);
    } else {
        const float* xr = D.X32 + (int64_t)i * D.ldx;
        for (int l = 0; l < D.d; ++l) acc = __fma_rn((double)u[l], (double)xr[l], acc);
    }
    return acc;
}

// Exact median / MAD / MAD_+ of one direction's keys y (after the projection pass) and the
// depth, by its group q of GS threads.  The selection runs on the FP32 keys and yields the points
// holding the wanted order statistics (ties broken by point index); the depth is then formed from
// FP64 projections of those few points and the FP64 y_z (yzv).
//   median  the bucket run of ranks k1, k2 (from the key histogram H) is gathered and ranked;
//   D_P     in the same gather pass, two runs L, R placed symmetrically about the median run at the
//           bucket distance where the window count reaches the MAD rank; after the median is known
//           their deviations are ranked, and the result is accepted only when every key between the
//           runs deviates no more and every key outside no less than the picked values (else a
//           |y - med| histogram pass decides);
//   D_AP    in the same gather pass, the run of the MAD_+ ranks guessed for no key tying the median.
// Runs that overflow the gather buffer fall back to iterated bucket selection.
template <int GS, class K>
__device__ __forceinline__ void select_dir(const Grp<GS>& q, const K& y, Ctl& C, unsigned* H, float* B0, int* I0,
                                           int n, bool ap, const float* u, const DsDev& D, double yzv, int64_t roff,
                                           ResDev* __restrict__ res, int* err)
{
    const int g = q.g;
    float* B1 = B0 + CAP;   // MAD_+ guess run (D_AP) or the L, R runs (D_P); B0 holds the median run
    int* I1 = I0 + CAP;
    const float sc = C.sc_y[g], of = C.off_y[g];
    const int k1 = (n - 1) / 2, k2 = n / 2;
    const int n4 = n & ~3;
    const float qnan = __int_as_float(0x7FC00000);
    constexpr int OFF = 1 << 30;   // a run start no bucket test can reach

    int ba, ca, bb, cb;
    gfind(q, H, k1, k2, C, ba, ca, bb, cb);
    const int c_lo0 = ca, cnt0 = cb + (int)H[bb] - ca;
    int fb = cnt0 > CAP ? 1 : 0;   // 1: fall back for every statistic, 2: only for the spread
    // second gathered set: buckets b with |2b - c2| in [dl2, dl2 + dw2]
    int c2 = 0, dl2 = OFF, dw2 = 0, c_lo1 = 0, cnt1 = 0, c_in = 0;
    const int npos_guess = (n & 1) ? (n - 1) / 2 : n / 2;
    if (ap && npos_guess > 0) {
        const int base = n - npos_guess;
        int b3, c3, b4, c4;
        gfind(q, H, base + (npos_guess - 1) / 2, base + npos_guess / 2, C, b3, c3, b4, c4);
        c_lo1 = c3;
        cnt1 = c4 + (int)H[b4] - c3;
        if (cnt1 > CAP) fb = 1;
        c2 = 2 * b3 + (b4 - b3);   // the run [b3, b4]
        dl2 = 0;
        dw2 = b4 - b3;
    } else if (!ap && !fb) {
        gprefix(q, H, C);   // H: inclusive prefix counts from here on (the fallbacks rebuild it)
        // smallest s with more than k2 keys in the buckets [ba - s, bb + s]
        if (q.t == 0) C.f_b1[g] = NB;
        q.sync();
        constexpr int PER = NB / GS;
#pragma unroll 1
        for (int k = 0; k < PER; ++k) {
            const int s = q.t * PER + k;
            const int hi = bb + s < NB - 1 ? bb + s : NB - 1, lo = ba - s;
            const int c = (int)H[hi] - (lo >= 1 ? (int)H[lo - 1] : 0);
            if (c > k2) {
                atomicMin(&C.f_b1[g], s);
                break;
            }
        }
        q.sync();
        const int ss = C.f_b1[g];
        q.sync();
        // keys deviating by about the MAD sit within w + 1 buckets of distance ss from the median run
        const int w = bb - ba + 1;
        const int L0 = ba - ss - w - 1, L1 = ba - ss + w + 1, R0 = bb + ss - w - 1, R1 = bb + ss + w + 1;
        if (ss >= w + 2 && L0 >= 1 && R1 <= NB - 2) {
            const int cl = (int)(H[L1] - H[L0 - 1]) + (int)(H[R1] - H[R0 - 1]);
            if (cl <= CAP) {
                cnt1 = cl;
                c_in = (int)(H[R0 - 1] - H[L1]);
                c2 = ba + bb;
                dl2 = 2 * ss - w - 3;
                dw2 = 4 * w + 4;
            }
        }
    }
    float m1 = qnan, m2 = qnan, p1 = 0.f, p2 = 0.f;
    int im1 = -1, im2 = -1, ip1 = -1, ip2 = -1;
    int npos = 0;
    if (!fb) {
        if (q.t < 2) C.fill[g][q.t] = 0;
        q.sync();
        const int bl0 = ba, bw0 = bb - ba;
        auto gather = [&](float v, int i) {
            const int b = bucket_fma(v, sc, of);
            if ((unsigned)(b - bl0) <= (unsigned)bw0) {
                const int pos = atomicAdd(&C.fill[g][0], 1);
                if (pos < CAP) {
                    B0[pos] = v;
                    I0[pos] = i;
                }
            }
            if ((unsigned)(abs(2 * b - c2) - dl2) <= (unsigned)dw2) {
                const int pos = atomicAdd(&C.fill[g][1], 1);
                if (pos < CAP) {
                    B1[pos] = v;
                    I1[pos] = i;
                }
            }
        };
        for (int i = 4 * q.t; i < n4; i += 4 * GS) {
            const float4 y4 = y.get4(i);
            gather(y4.x, i);
            gather(y4.y, i + 1);
            gather(y4.z, i + 2);
            gather(y4.w, i + 3);
        }
        for (int i = n4 + q.t; i < n; i += GS) gather(y.get(i), i);
        q.sync();
        gpick(q, B0, I0, cnt0, k1 - c_lo0, k2 - c_lo0, C, m1, m2, im1, im2);
        if (ap) {
            // #(y <= med) = #(y <= m1): keys below the run plus gathered keys <= m1
            int c = 0;
            for (int t = q.t; t < cnt0; t += GS) c += (B0[t] <= m1);
            const int nle = c_lo0 + gsum(q, c, C);
            npos = n - nle;
            if (npos > 0) {
                const int s3 = nle + (npos - 1) / 2 - c_lo1, s4 = nle + npos / 2 - c_lo1;
                if (s3 < 0 || s4 >= cnt1)
                    fb = 2;   // the positive count differed from the guess
                else
                    gpick(q, B1, I1, cnt1, s3, s4, C, p1, p2, ip1, ip2);
            }
        } else {
            const float m = __fmul_rn(__fadd_rn(m1, m2), 0.5f);
            bool ok = dl2 != OFF;
            if (ok) {
                // L keys lie below m1 <= m, R keys above m2 >= m; deviations in place, and the extremes of each run
                float lmin = FLT_MAX, lmax = -FLT_MAX, rmin = FLT_MAX, rmax = -FLT_MAX;
                for (int t = q.t; t < cnt1; t += GS) {
                    const float v = B1[t];
                    if (v < m) {
                        lmin = fminf(lmin, v);
                        lmax = fmaxf(lmax, v);
                    } else {
                        rmin = fminf(rmin, v);
                        rmax = fmaxf(rmax, v);
                    }
                    B1[t] = fabsf(__fsub_rn(v, m));
                }
                float la, lb, ra, rb;
                gminmax(q, lmin, lmax, C, la, lb);
                gminmax(q, rmin, rmax, C, ra, rb);
                const int s1 = k1 - c_in, s2 = k2 - c_in;
                ok = lb > -FLT_MAX && ra < FLT_MAX && s1 >= 0 && s2 < cnt1;
                if (ok) {
                    gpick(q, B1, I1, cnt1, s1, s2, C, p1, p2, ip1, ip2);
                    // keys between the runs lie in (max L, min R), keys outside below min L or above max R
                    const float inner = fmaxf(__fsub_rn(m, lb), __fsub_rn(ra, m));
                    const float outer = fminf(__fsub_rn(m, la), __fsub_rn(rb, m));
                    ok = inner <= p1 && outer >= p2;
                }
            }
            if (!ok) {
                // |y - med| histogram over [0, 4 sigma_u] (edge bucket clamps), gather, ranks
                float dmax = D.cov ? 4.0f * C.scale[g] : 0.0f;
                const float hard =
                    __fmul_rn(__fadd_rn(D.rc, fabsf(m - C.lo_b[g] - 0.5f * (float)NB / sc)), 1.0001f);
                if (!(dmax > 0.0f) || dmax > hard) dmax = hard;
                if (!(dmax > 0.0f)) dmax = 1.0f;
                const float scd = __fdiv_rn((float)NB, dmax);
                for (int b = q.t; b < NB / 4; b += GS) reinterpret_cast<uint4*>(H)[b] = make_uint4(0u, 0u, 0u, 0u);
                q.sync();
                for (int i = 4 * q.t; i < n4; i += 4 * GS) {
                    const float4 y4 = y.get4(i);
                    atomicAdd(&H[bucket_fma(fabsf(__fsub_rn(y4.x, m)), scd, 0.0f)], 1u);
                    atomicAdd(&H[bucket_fma(fabsf(__fsub_rn(y4.y, m)), scd, 0.0f)], 1u);
                    atomicAdd(&H[bucket_fma(fabsf(__fsub_rn(y4.z, m)), scd, 0.0f)], 1u);
                    atomicAdd(&H[bucket_fma(fabsf(__fsub_rn(y4.w, m)), scd, 0.0f)], 1u);
                }
                for (int i = n4 + q.t; i < n; i += GS)
                    atomicAdd(&H[bucket_fma(fabsf(__fsub_rn(y.get(i), m)), scd, 0.0f)], 1u);
                q.sync();
                int da, dca, db, dcb;
                gfind(q, H, k1, k2, C, da, dca, db, dcb);
                const int cntd = dcb + (int)H[db] - dca;
                if (cntd > CAP) {
                    fb = 2;
                } else {
                    if (q.t == 0) C.fill[g][1] = 0;
                    q.sync();
                    const int bwd = db - da;
                    auto gd = [&](float v, int i) {
                        const float dv = fabsf(__fsub_rn(v, m));
                        const int b = bucket_fma(dv, scd, 0.0f);
                        if ((unsigned)(b - da) <= (unsigned)bwd) {
                            const int pos = atomicAdd(&C.fill[g][1], 1);
                            if (pos < CAP) {
                                B1[pos] = dv;
                                I1[pos] = i;
                            }
                        }
                    };
                    for (int i = 4 * q.t; i < n4; i += 4 * GS) {
                        const float4 y4 = y.get4(i);
                        gd(y4.x, i);
                        gd(y4.y, i + 1);
                        gd(y4.z, i + 2);
                        gd(y4.w, i + 3);
                    }
                    for (int i = n4 + q.t; i < n; i += GS) gd(y.get(i), i);
                    q.sync();
                    gpick(q, B1, I1, cntd, k1 - dca, k2 - dca, C, p1, p2, ip1, ip2);
                }
            }
        }
    }

    // ---- fallback: iterated bucket selection over this direction's keys ----------------
    if (fb) {
        float kl = FLT_MAX, kh = -FLT_MAX;
        for (int i = q.t; i < n; i += GS) {
            const float v = y.get(i);
            kl = fminf(kl, v);
            kh = fmaxf(kh, v);
        }
        gminmax(q, kl, kh, C, kl, kh);
        unsigned* HF = H;
        float* BF = B0;   // FB_CAP values: B0 and B1
        int* IF = I0;     // and their indices: I0 and I1
        if (fb == 1)
            gselect(q, [&](int i) { return y.get(i); }, n, k1, k2, kl, kh, HF, BF, IF, C, m1, m2, im1, im2, err);
        if (ap) {
            int c = 0;
            for (int i = q.t; i < n; i += GS) c += (y.get(i) <= m1);
            const int nle = gsum(q, c, C);
            npos = n - nle;
            ip1 = ip2 = -1;
            if (npos > 0)
                gselect(q, [&](int i) { return y.get(i); }, n, nle + (npos - 1) / 2, nle + npos / 2, kl, kh, HF, BF,
                        IF, C, p1, p2, ip1, ip2, err);
        } else {
            const float m = __fmul_rn(__fadd_rn(m1, m2), 0.5f);
            const float dmax = fmaxf(fabsf(__fsub_rn(kl, m)), fabsf(__fsub_rn(kh, m)));
            gselect(q, [&](int i) { return fabsf(__fsub_rn(y.get(i), m)); }, n, k1, k2, 0.0f, dmax, HF, BF, IF, C,
                    p1, p2, ip1, ip2, err);
        }
    }

    // ---- depth from FP64 projections of the selected points --------------------------------
    const int sel = q.t == 0 ? im1 : (q.t == 1 ? im2 : (q.t == 2 ? ip1 : ip2));
    if (q.t < 4) C.y64[g][q.t] = sel >= 0 ? proj64(D, u, sel) : 0.0;
    q.sync();
    if (q.t == 0) {
        const double* Y = C.y64[g];
        double depth = __longlong_as_double(0x7FF8000000000000LL);   // a failed selection (error flag set)
        if (im1 >= 0 && im2 >= 0) {
            const double med = (Y[0] + Y[1]) * 0.5;
            if (ap) {
                double madp = 0.0;
                if (npos > 0) madp = ip1 >= 0 && ip2 >= 0 ? fmax(((Y[2] - med) + (Y[3] - med)) * 0.5, 0.0) : depth;
                depth = depth_from(yzv - med > 0.0 ? yzv - med : 0.0, madp);
            } else if (ip1 >= 0 && ip2 >= 0) {
                depth = depth_from(fabs(yzv - med), (fabs(Y[2] - med) + fabs(Y[3] - med)) * 0.5);
            }
        }
        res[roff + g] = ResDev{depth, -1};
    }
}

// Every live direction of the CTA: group g of cta_threads<G>() / G threads handles direction g alone,
// on its keys in shared memory or (STREAM) on keys formed by launch_pdap_keys in global memory (kin), else
// on keys recomputed from X.
template <int G, int DP4, bool STREAM>
__device__ __forceinline__ void select_dirs(Ctl& C, const float* keys, const float* uS, unsigned* hist, float* buf,
                                            int* ibuf, int n, int npad, bool ap, const DsDev& D, int GA,
                                            const double* yz, int64_t roff, ResDev* __restrict__ res, int* err,
                                            const float* kin)
{
    constexpr int GS = cta_threads<G>() / G;   // threads per direction group
    const int tid = threadIdx.x;
    const Grp<GS> q{tid / GS, tid % GS};
    const int g = q.g;
    if (g >= GA) return;   // inert direction (no CTA-wide barrier follows)
    unsigned* H = hist + g * NB;
    float* B0 = buf + (size_t)(2 * g) * CAP;   // two gather runs; FB_CAP = 2 * CAP for the fallback
    int* I0 = ibuf + (size_t)(2 * g) * CAP;    // the point index of every gathered key
    const float* u = uS + (size_t)g * D.ldx;
    const double yzv = yz[roff + g];
    if (STREAM && kin) {
        const KeysArray y{kin + ((size_t)blockIdx.x * G + g) * npad};
        select_dir<GS>(q, y, C, H, B0, I0, n, ap, u, D, yzv, roff, res, err);
    } else if (STREAM) {
        const KeysRecomputed<DP4> y{D.X32, u, D.ldx, DP4 ? DP4 : ((D.d + 3) & ~3)};
        select_dir<GS>(q, y, C, H, B0, I0, n, ap, u, D, yzv, roff, res, err);
    } else {
        const KeysArray y{keys + (size_t)g * npad};
        select_dir<GS>(q, y, C, H, B0, I0, n, ap, u, D, yzv, roff, res, err);
    }
}

// G: directions per CTA (compile time); DP4: d rounded up to 4 when <= 16 (the
// directions are then held in registers), 0 for any d; STREAM: no keys in shared
// memory, every pass reads them from kin or recomputes them from X.
// kin: optional precomputed keys, G x npad per task in launch order (launch_pdap_keys), read instead of
// projecting
template <int G, int DP4, bool STREAM>
__global__ void __launch_bounds__(cta_threads<G>(), (G >= 4 ? 1 : 2)) k_pdap2(const TaskDev* __restrict__ tasks, const SlotDev* __restrict__ slots,
                                                 const DsDev* __restrict__ dsets, const float* __restrict__ U,
                                                 const double* __restrict__ yz, ResDev* __restrict__ res, int* err,
                                                 const float* __restrict__ kin)
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
    float* keys = sm;                                          // G x npad (none when STREAM)
    float* uS = keys + (STREAM ? (size_t)0 : (size_t)G * npad);   // G x ldx
    unsigned* hist = reinterpret_cast<unsigned*>(uS + (size_t)G * ldx);   // G x NB
    float* buf = reinterpret_cast<float*>(hist + (size_t)G * NB);        // G x 2 x CAP
    int* ibuf = reinterpret_cast<int*>(buf + (size_t)G * 2 * CAP);       // G x 2 x CAP

    const int GA = T.nj;   // live directions; groups GA..G-1 are inert
    constexpr int NTK = cta_threads<G>();
    for (int e = tid; e < G * ldx; e += NTK) uS[e] = (e / ldx < GA) ? U[S.uoff + (int64_t)T.j0 * ldx + e] : 0.0f;
    for (int e = tid; e < G * NB / 4; e += NTK) reinterpret_cast<uint4*>(hist)[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    // per-direction bucket range: the centre's projection +- 5 sigma_u (sigma_u^2 = u' Cov u),
    // or +- the radius about the centre when no covariance is kept.  Keys outside the range go
    // to the edge buckets, which keeps the bucket map monotone.  One warp per direction: lanes
    // take rows of Cov (the range is a heuristic, so its summation order is free); y_z keeps the
    // keys' own arithmetic (one lane, sequential FMAs).
    if ((tid >> 5) < G) {
        const int g = tid >> 5, lane = tid & 31;
        const float* u = uS + g * ldx;
        float yc = 0.0f, qf = 0.0f;
        for (int r = lane; r < d; r += 32) yc = fmaf(u[r], D.center[r], yc);
        if (D.cov) {
            // lanes stride over the d x d entries, so the covariance loads are independent of each other
            for (int e = lane; e < d * d; e += 32) {
                const int r = e / d, c2 = e - r * d;
                qf = fmaf(D.cov[e], __fmul_rn(u[r], u[c2]), qf);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            yc += __shfl_xor_sync(0xFFFFFFFFu, yc, o);
            qf += __shfl_xor_sync(0xFFFFFFFFu, qf, o);
        }
        if (lane == 0) {
            float half = D.rc * 1.0001f;
            if (D.cov) {
                const float sg = sqrtf(fmaxf(qf, 0.0f));
                if (sg > 0.0f && 5.0f * sg < half) half = 5.0f * sg;
                C.scale[g] = sg;   // kept for the deviation range
            } else {
                C.scale[g] = half;
            }
            if (!(half > 0.0f)) half = fmaxf(fabsf(yc), 1.0f);
            C.lo_b[g] = yc - half;
            C.sc_y[g] = __fdiv_rn((float)NB, __fadd_rn(half, half));
            C.off_y[g] = __fmul_rn(-C.lo_b[g], C.sc_y[g]);
        }
    }
    __syncthreads();

    // ---- pass A (whole CTA): keys + bucket counts ---------------------------------------
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
                if (!STREAM) keys[(size_t)g * npad + i] = acc[g];
                atomicAdd(&hist[g * NB + bucket_fma(acc[g], sc[g], of[g])], 1u);
            }
        };
        if (kin) {
            // keys formed by k_keys (same arithmetic as the projection below): count (and copy unless STREAM)
            const float4* src = reinterpret_cast<const float4*>(kin + (size_t)blockIdx.x * G * npad);
            for (int e = tid; e < G * npad / 4; e += NTK) {
                const int g = e / (npad / 4), i = 4 * (e - g * (npad / 4));
                if (g >= GA) continue;
                const float4 k4 = src[e];
                const float kv[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    if (i + h < n) {
                        if (!STREAM) keys[(size_t)g * npad + i + h] = kv[h];
                        atomicAdd(&hist[g * NB + bucket_fma(kv[h], sc[g], of[g])], 1u);
                    }
                }
            }
        } else if (G == 4 && DP4 > 0) {
            // two adjacent lanes per point, each forming the keys of two directions: the row load is
            // coalesced within the warp and each lane holds only two direction vectors
            constexpr int D4 = DP4 > 0 ? DP4 : 4;
            const int pair = tid & 1;
            float ua[D4], ub[D4];
#pragma unroll
            for (int l = 0; l < D4; ++l) {
                ua[l] = uS[(2 * pair) * ldx + l];
                ub[l] = uS[(2 * pair + 1) * ldx + l];
            }
            const float sca = sc[2 * pair], ofa = of[2 * pair], scb = sc[2 * pair + 1], ofb = of[2 * pair + 1];
            for (int i = tid >> 1; i < n; i += NTK / 2) {
                const float4* xr = reinterpret_cast<const float4*>(D.X32 + (int64_t)i * ldx);
                float xv[D4];
#pragma unroll
                for (int c = 0; c < D4 / 4; ++c) {
                    const float4 t4 = xr[c];
                    xv[4 * c] = t4.x;
                    xv[4 * c + 1] = t4.y;
                    xv[4 * c + 2] = t4.z;
                    xv[4 * c + 3] = t4.w;
                }
                const float ka = key_halves<D4>(ua, xv), kb = key_halves<D4>(ub, xv);
                if (!STREAM) keys[(size_t)(2 * pair) * npad + i] = ka;
                atomicAdd(&hist[(2 * pair) * NB + bucket_fma(ka, sca, ofa)], 1u);
                if (!STREAM) keys[(size_t)(2 * pair + 1) * npad + i] = kb;
                atomicAdd(&hist[(2 * pair + 1) * NB + bucket_fma(kb, scb, ofb)], 1u);
            }
        } else if (DP4 > 0) {
            float4 ur[G][DP4 > 0 ? DP4 / 4 : 1];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int c = 0; c < DP4 / 4; ++c) ur[g][c] = *reinterpret_cast<const float4*>(uS + g * ldx + 4 * c);
            // two points per iteration: both rows' loads are in flight together
            for (int i = tid; i < n; i += 2 * NTK) {
                const int i2 = i + NTK;
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
                for (int g = 0; g < G; ++g) {
                    // key_halves on the register copies (one row's dims as plain floats)
                    float uu[DP4 > 0 ? DP4 : 4], xa_[DP4 > 0 ? DP4 : 4], xb_[DP4 > 0 ? DP4 : 4];
#pragma unroll
                    for (int c = 0; c < DP4 / 4; ++c) {
                        uu[4 * c] = ur[g][c].x;
                        uu[4 * c + 1] = ur[g][c].y;
                        uu[4 * c + 2] = ur[g][c].z;
                        uu[4 * c + 3] = ur[g][c].w;
                        xa_[4 * c] = va[c].x;
                        xa_[4 * c + 1] = va[c].y;
                        xa_[4 * c + 2] = va[c].z;
                        xa_[4 * c + 3] = va[c].w;
                        xb_[4 * c] = vb[c].x;
                        xb_[4 * c + 1] = vb[c].y;
                        xb_[4 * c + 2] = vb[c].z;
                        xb_[4 * c + 3] = vb[c].w;
                    }
                    acc[g] = key_halves<(DP4 > 0 ? DP4 : 4)>(uu, xa_);
                    acc2[g] = key_halves<(DP4 > 0 ? DP4 : 4)>(uu, xb_);
                }
                emit(i, acc);
                if (two) emit(i2, acc2);
            }
        } else {
            for (int i = tid; i < n; i += NTK) {
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

    select_dirs<G, DP4, STREAM>(C, keys, uS, hist, buf, ibuf, n, npad, ap, D, GA, yz, S.roff + T.j0, res, err, kin);
}

}  // namespace

size_t pdap_smem_bytes(int n, int group, int ldx, bool stream)
{
    const size_t npad = stream ? 0 : ((size_t)n + 3) & ~(size_t)3;
    return sizeof(float) * ((size_t)group * npad + (size_t)group * ldx) + sizeof(unsigned) * (size_t)group * NB +
           (sizeof(float) + sizeof(int)) * (size_t)group * 2 * CAP;
}

size_t pdap_smem_limit()
{
    // opt-in maximum per CTA (227 KB) minus the kernels' static blocks
    return 232448 - sizeof(Ctl) - 64 - 256;
}

size_t pdap_two_per_sm_limit()
{
    // 228 KB per SM shared by two CTAs, each also holding 1 KB of reserved and ~1 KB of static memory
    return 112 * 1024;
}

int pdap_max_group(int n, int ldx, int m, int d, bool keys_in)
{
    // G in {1, 2, 4}: the largest G that fits two CTAs per SM when that is at least 2, else the
    // largest that fits one CTA per SM.  Exception: for d > 16 with keys formed inside the kernel
    // the projection pass re-reads X (4 d bytes per point) for every G directions, so there the
    // largest G that fits wins (measured at n = 10,000: d = 50 1.27x, d = 150 1.68x faster with
    // G = 4 than G = 2); with keys from k_keys the usual rule holds again.
    const size_t one = pdap_smem_limit(), two = pdap_two_per_sm_limit();
    int g_one = 0, g_two = 0;
    for (int g = 1; g <= MAXG && g <= m; g *= 2) {
        const size_t need = pdap_smem_bytes(n, g, ldx);
        if (need <= one) g_one = g;
        if (need <= two) g_two = g;
    }
    if (pdap_dp4_class(d) == 0 && !keys_in) return g_one;
    if (g_two >= 2) return g_two;
    return g_one;
}

// Keys of a block of tasks (G directions each, all of one dataset) for every point, as a tiled FP32
// GEMM: keys[(t * G + g) * npad + i] = u_{t,g}'x_i, each key one sequential FMA chain over the dims
// (the selection kernel's own arithmetic for d > 16, and y_z's), so results do not depend on which
// kernel formed the keys.  CTA tile: 128 points x 128 directions, 256 threads of 8 x 8 outputs, the
// dims staged 16 at a time in shared memory.
constexpr int KT_P = 128, KT_D = 128, KT_K = 16;

__global__ void __launch_bounds__(256) k_keys(const TaskDev* __restrict__ tasks, int ntasks, int G,
                                              const SlotDev* __restrict__ slots, const DsDev* __restrict__ dsets,
                                              const float* __restrict__ U, float* __restrict__ keys, int npad)
{
    __shared__ __align__(16) float Xs[KT_K][KT_P + 4];   // [dim][point]
    __shared__ __align__(16) float Us[KT_K][KT_D + 4];   // [dim][direction]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const DsDev D = dsets[slots[tasks[0].slot].ds];
    const int n = (int)D.n, ldx = D.ldx, dp4 = (D.d + 3) & ~3;
    const int i0 = blockIdx.x * KT_P, r0 = blockIdx.y * KT_D;
    // staging: thread tid loads 8 dims of point row tid / 2 and 8 dims of direction row tid / 2
    const int lr = tid >> 1, lh = (tid & 1) * 8;
    const float* urow = nullptr;
    {
        const int r = r0 + lr, t = r / G, g = r - t * G;
        if (t < ntasks && g < tasks[t].nj) {
            const TaskDev T = tasks[t];
            urow = U + slots[T.slot].uoff + (int64_t)(T.j0 + g) * ldx;
        }
    }
    const float* xrow = (i0 + lr < n) ? D.X32 + (int64_t)(i0 + lr) * ldx : nullptr;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
    for (int k0 = 0; k0 < dp4; k0 += KT_K) {
        // zero beyond the row (rows are zero-padded to ldx, so the extra terms add exact zeros)
#pragma unroll
        for (int h = 0; h < 8; h += 4) {
            const int l = k0 + lh + h;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f), w = v;
            if (xrow && l + 4 <= ldx) v = *reinterpret_cast<const float4*>(xrow + l);
            if (urow && l + 4 <= ldx) w = *reinterpret_cast<const float4*>(urow + l);
            Xs[lh + h][lr] = v.x;
            Xs[lh + h + 1][lr] = v.y;
            Xs[lh + h + 2][lr] = v.z;
            Xs[lh + h + 3][lr] = v.w;
            Us[lh + h][lr] = w.x;
            Us[lh + h + 1][lr] = w.y;
            Us[lh + h + 2][lr] = w.z;
            Us[lh + h + 3][lr] = w.w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KT_K; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Xs[kk][tx * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Xs[kk][tx * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Us[kk][ty * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Us[kk][ty * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(bv[c], av[a], acc[a][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int r = r0 + ty * 8 + c, t = r / G, g = r - t * G;
        if (t >= ntasks || g >= tasks[t].nj) continue;
        float* out = keys + (size_t)r * npad + i0 + tx * 8;
        if (i0 + tx * 8 + 4 <= npad) *reinterpret_cast<float4*>(out) = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
        if (i0 + tx * 8 + 8 <= npad)
            *reinterpret_cast<float4*>(out + 4) = make_float4(acc[4][c], acc[5][c], acc[6][c], acc[7][c]);
    }
}

// Keys for d <= 16 (DP4 = d rounded up to 4) with the selection kernel's own two-half-chain arithmetic
// (key_halves), same layout as k_keys: keys[(t * G + g) * npad + i].  CTA: 256 points x 16 directions,
// one point row in registers per thread, the directions in shared memory, coalesced key writes.
constexpr int KH_P = 256, KH_D = 16;

template <int DP4>
__global__ void __launch_bounds__(KH_P) k_keys_halves(const TaskDev* __restrict__ tasks, int ntasks, int G,
                                                      const SlotDev* __restrict__ slots,
                                                      const DsDev* __restrict__ dsets, const float* __restrict__ U,
                                                      float* __restrict__ keys, int npad)
{
    __shared__ __align__(16) float Us[KH_D][DP4];
    __shared__ int live[KH_D];
    const DsDev D = dsets[slots[tasks[0].slot].ds];
    const int n = (int)D.n, ldx = D.ldx;
    const int r0 = blockIdx.y * KH_D;
    for (int e = threadIdx.x; e < KH_D * DP4; e += KH_P) {
        const int rr = e / DP4, l = e - rr * DP4, r = r0 + rr, t = r / G, g = r - t * G;
        float v = 0.0f;
        if (t < ntasks && g < tasks[t].nj) v = U[slots[tasks[t].slot].uoff + (int64_t)(tasks[t].j0 + g) * ldx + l];
        Us[rr][l] = v;
    }
    if (threadIdx.x < KH_D) {
        const int r = r0 + threadIdx.x, t = r / G, g = r - t * G;
        live[threadIdx.x] = t < ntasks && g < tasks[t].nj;
    }
    __syncthreads();
    const int i = blockIdx.x * KH_P + threadIdx.x;
    if (i >= n) return;
    const float4* xr = reinterpret_cast<const float4*>(D.X32 + (int64_t)i * ldx);
    float xv[DP4];
#pragma unroll
    for (int c = 0; c < DP4 / 4; ++c) {
        const float4 t4 = xr[c];
        xv[4 * c] = t4.x;
        xv[4 * c + 1] = t4.y;
        xv[4 * c + 2] = t4.z;
        xv[4 * c + 3] = t4.w;
    }
#pragma unroll 4
    for (int rr = 0; rr < KH_D; ++rr)
        if (live[rr]) keys[(size_t)(r0 + rr) * npad + i] = key_halves<DP4>(Us[rr], xv);
}

template <int G, int DP4, bool STREAM>
static cudaError_t launch_t(const TaskDev* tasks, int ntasks, size_t smem, const SlotDev* slots, const DsDev* ds,
                            const float* U, const double* yz, ResDev* res, int* err, const float* kin, cudaStream_t st)
{
    cudaError_t e =
        cudaFuncSetAttribute(k_pdap2<G, DP4, STREAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();   // do not leave the failure pending for an unrelated later call
        return e;
    }
    k_pdap2<G, DP4, STREAM><<<ntasks, cta_threads<G>(), smem, st>>>(tasks, slots, ds, U, yz, res, err, kin);
    return cudaGetLastError();
}

template <int G, bool STREAM>
static cudaError_t launch_g(int dp4, const TaskDev* tasks, int ntasks, size_t smem, const SlotDev* slots,
                            const DsDev* ds, const float* U, const double* yz, ResDev* res, int* err, const float* kin,
                            cudaStream_t st)
{
    switch (dp4) {
    case 4: return launch_t<G, 4, STREAM>(tasks, ntasks, smem, slots, ds, U, yz, res, err, kin, st);
    case 8: return launch_t<G, 8, STREAM>(tasks, ntasks, smem, slots, ds, U, yz, res, err, kin, st);
    case 12: return launch_t<G, 12, STREAM>(tasks, ntasks, smem, slots, ds, U, yz, res, err, kin, st);
    case 16: return launch_t<G, 16, STREAM>(tasks, ntasks, smem, slots, ds, U, yz, res, err, kin, st);
    default: return launch_t<G, 0, STREAM>(tasks, ntasks, smem, slots, ds, U, yz, res, err, kin, st);
    }
}

int pdap_dp4_class(int d)
{
    const int dp4 = (d + 3) & ~3;
    return dp4 <= 16 ? dp4 : 0;
}

cudaError_t launch_pdap(const TaskDev* tasks, int ntasks, size_t smem, int group, int variant, const SlotDev* slots,
                        const DsDev* ds, const float* U, const double* yz, ResDev* res, int* err, cudaStream_t st,
                        const float* kin)
{
    if (ntasks <= 0) return cudaSuccess;
    if (smem > pdap_smem_limit()) return cudaErrorInvalidValue;
    const int dp4 = variant & ~PDAP_STREAM;
    if (variant & PDAP_STREAM) {
        if (group != PDAP_STREAM_GROUP) return cudaErrorInvalidValue;
        return launch_g<PDAP_STREAM_GROUP, true>(dp4, tasks, ntasks, smem, slots, ds, U, yz, res, err, kin, st);
    }
    switch (group) {
    case 1: return launch_g<1, false>(dp4, tasks, ntasks, smem, slots, ds, U, yz, res, err, kin, st);
    case 2: return launch_g<2, false>(dp4, tasks, ntasks, smem, slots, ds, U, yz, res, err, kin, st);
    case 4: return launch_g<4, false>(dp4, tasks, ntasks, smem, slots, ds, U, yz, res, err, kin, st);
    default: return cudaErrorInvalidValue;
    }
}

PdapShape pdap_shape(int n, int ldx, int m, int d, int group)
{
    PdapShape s{};
    const int dp4 = pdap_dp4_class(d);
    int G = group;
    if (G && (G > m || pdap_smem_bytes(n, G, ldx) > pdap_smem_limit())) G = 0;
    if (!G) G = pdap_max_group(n, ldx, m, d, dp4 == 0);
    if (G) {
        s.group = G;
        s.variant = dp4;
        s.smem = pdap_smem_bytes(n, G, ldx);
        s.keys_gemm = dp4 == 0;
    } else {
        s.group = PDAP_STREAM_GROUP;
        s.variant = dp4 | PDAP_STREAM;
        s.smem = pdap_smem_bytes(n, PDAP_STREAM_GROUP, ldx, true);
        // the selection passes read keys formed once (k_keys, or k_keys_halves for d <= 16) instead of
        // re-forming the dot products from X at every pass
        s.keys_gemm = true;
    }
    return s;
}

size_t pdap_keys_bytes(int n, int group, int ntasks)
{
    return sizeof(float) * (size_t)ntasks * group * (((size_t)n + 3) & ~(size_t)3);
}

cudaError_t launch_pdap_keys(const TaskDev* tasks, int ntasks, int group, const SlotDev* slots, const DsDev* ds,
                             const DsDev& ds_host, const float* U, float* keys, cudaStream_t st)
{
    if (ntasks <= 0) return cudaSuccess;
    if (ds_host.n < 1 || ds_host.n > PDAP_MAX_N) return cudaErrorInvalidValue;
    const int npad = (int)((ds_host.n + 3) & ~3LL);
    const int dp4 = pdap_dp4_class(ds_host.d);
    if (dp4 > 0) {
        const dim3 grid((unsigned)((ds_host.n + KH_P - 1) / KH_P), (unsigned)((ntasks * group + KH_D - 1) / KH_D));
        switch (dp4) {
        case 4: k_keys_halves<4><<<grid, KH_P, 0, st>>>(tasks, ntasks, group, slots, ds, U, keys, npad); break;
        case 8: k_keys_halves<8><<<grid, KH_P, 0, st>>>(tasks, ntasks, group, slots, ds, U, keys, npad); break;
        case 12: k_keys_halves<12><<<grid, KH_P, 0, st>>>(tasks, ntasks, group, slots, ds, U, keys, npad); break;
        default: k_keys_halves<16><<<grid, KH_P, 0, st>>>(tasks, ntasks, group, slots, ds, U, keys, npad); break;
        }
        return cudaGetLastError();
    }
    const dim3 grid((unsigned)((ds_host.n + KT_P - 1) / KT_P), (unsigned)((ntasks * group + KT_D - 1) / KT_D));
    k_keys<<<grid, 256, 0, st>>>(tasks, ntasks, group, slots, ds, U, keys, npad);
    return cudaGetLastError();
}

}  // namespace rrs
