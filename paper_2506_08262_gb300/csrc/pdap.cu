// Projection depth D_P and asymmetric projection depth D_AP (Sec. 2) for a block
// of directions: y_i = u'x_i in FP32, exact order statistics (median, MAD,
// MAD_+) of the FP32 keys, whose points a second kernel (k_pdap_finish)
// re-projects in FP64 to form the depth.
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
#include <limits.h>
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
constexpr int CAP = 256;     // gathered keys per direction: the median run (and the D_AP MAD_+ run)
constexpr int CAP1 = 512;    // second gather buffer: the D_AP MAD_+ run or the D_P MAD runs L, R
constexpr int CAP1H = (NB - 256) / 2;   // D_P runs too large for it: pairs in the histogram area (after 256 counters)
constexpr int MAXG = 4;
// Stride of the resident keys of one direction in shared memory: n rounded up to 32 floats (128 bytes)
__host__ __device__ constexpr int pdap_key_stride(int n) { return (n + 31) & ~31; }
constexpr int FB_NB = NB;    // fallback histogram (reuses the bucket area)
constexpr int FB_CAP = CAP + CAP1;  // fallback gather buffer: a direction's two gather areas

// Per-direction constants and per-group scratch: after the projection pass,
// group g (CTA threads / G) works on direction g alone and synchronises with
// the named barrier 1 + g, so the directions of a CTA never wait for each other.
struct Ctl {
    float lo_b[MAXG], sc_y[MAXG];      // bucket map of the keys: about (y - lo_b) * sc_y
    float off_y[MAXG];                 // -lo_b * sc_y + 2^23 (bucket_m offset)
    float scale[MAXG];                 // sigma_u (or the radius) of each direction
    int red[MAXG][NWARP];
    float fred[MAXG][2 * NWARP];
    int fill[MAXG][2];
    int f_b1[MAXG], f_c1[MAXG], f_b2[MAXG], f_c2[MAXG];   // bucket search results
    int fr_b[MAXG][4], fr_c[MAXG][4], fr_h[MAXG][4];      // gfindn: bucket, keys below, keys in it
    float pv1[MAXG], pv2[MAXG];                           // rank pick results
    int pi1[MAXG], pi2[MAXG];                             // their point indices
    int gn[MAXG];
    int gi[MAXG];                                         // smallest index of a tied run (fallback)
};

template <int GS>
struct Grp {
    int g, t;   // direction (group) index, thread index within the group
    __device__ __forceinline__ void sync() const
    {
        if constexpr (GS == 32)
            __syncwarp();   // one warp per direction: no named barrier needed
        else
            asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(GS) : "memory");
    }
};

template <int NBK = NB>
__device__ __forceinline__ int bucket(float y, float lo, float scale)
{
    // (y - lo) * scale, rounded once, truncated: monotone in y
    const int b = __float2int_rz(__fmul_rn(__fsub_rn(y, lo), scale));
    return b < 0 ? 0 : (b > NBK - 1 ? NBK - 1 : b);
}

// Bucket of the pass maps: y*sc + off rounded once, truncated (negatives saturate to 0),
// clamped to the last bucket.  Monotone non-decreasing in y.
template <int NBK = NB>
__device__ __forceinline__ int bucket_fma(float y, float sc, float off)
{
    const unsigned b = __float2uint_rz(__fmaf_rn(y, sc, off));
    return b < (unsigned)(NBK - 1) ? (int)b : NBK - 1;
}

// Bucket maps of k_pdap2: y*sc + off rounded once to an integer by the FMA itself.  o23 is off + 2^23,
// so a result r in [2^23, 2^24) is an integer and its float bits are MAGIC + (r - 2^23).  bucket_raw
// returns those bits as an int: non-decreasing in y for every result that is not a negative float, and
// every negative float is a negative int.  bucket_m clamps them to [0, NBK): no float-to-integer
// conversion, monotone non-decreasing in y.  A run of buckets [b1, b2] is the set of raw values in
// [raw_lo(b1), raw_hi(b2)] (signed comparisons), the edge buckets taking every value clamped into them.
constexpr int MAGIC = 0x4B000000;   // float bits of 2^23
constexpr float TWO23 = 8388608.0f;
__device__ __forceinline__ int bucket_raw(float y, float sc, float o23) { return __float_as_int(__fmaf_rn(y, sc, o23)); }
template <int NBK = NB>
__device__ __forceinline__ int bucket_m(float y, float sc, float o23)
{
    return min(max(bucket_raw(y, sc, o23), MAGIC), MAGIC + NBK - 1) - MAGIC;
}
template <int NBK = NB>
__device__ __forceinline__ int raw_lo(int b)
{
    return b <= 0 ? INT_MIN : MAGIC + b;
}
template <int NBK = NB>
__device__ __forceinline__ int raw_hi(int b)
{
    return b >= NBK - 1 ? INT_MAX : MAGIC + b;
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
template <int GS, class CT>
__device__ __forceinline__ int gsum(const Grp<GS>& q, int c, CT& C)
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
template <int GS, class CT>
__device__ void gminmax(const Grp<GS>& q, float lo, float hi, CT& C, float& olo, float& ohi)
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

// Group min and max of two pairs at once (one barrier round for both).
template <int GS, class CT>
__device__ __forceinline__ void gminmax2(const Grp<GS>& q, float& lo1, float& hi1, float& lo2, float& hi2, CT& C)
{
    constexpr int NW = GS / 32;   // at most 16: 4 NW values fit the 2 NWARP cells of fred
    static_assert(4 * NW <= 2 * NWARP, "gminmax2 scratch");
    lo1 = warp_min(lo1);
    hi1 = warp_max(hi1);
    lo2 = warp_min(lo2);
    hi2 = warp_max(hi2);
    const int w = q.t >> 5;
    if ((q.t & 31) == 0) {
        C.fred[q.g][w] = lo1;
        C.fred[q.g][NW + w] = hi1;
        C.fred[q.g][2 * NW + w] = lo2;
        C.fred[q.g][3 * NW + w] = hi2;
    }
    q.sync();
    lo1 = C.fred[q.g][0];
    hi1 = C.fred[q.g][NW];
    lo2 = C.fred[q.g][2 * NW];
    hi2 = C.fred[q.g][3 * NW];
#pragma unroll
    for (int i = 1; i < NW; ++i) {
        lo1 = fminf(lo1, C.fred[q.g][i]);
        hi1 = fmaxf(hi1, C.fred[q.g][NW + i]);
        lo2 = fminf(lo2, C.fred[q.g][2 * NW + i]);
        hi2 = fmaxf(hi2, C.fred[q.g][3 * NW + i]);
    }
    q.sync();
}

// Exclusive scan of h[0..NB) by the group; the bucket holding rank ra and the
// one holding rank rb (ra <= rb, both below the total), with the keys below each.
template <int GS, class CT, int NBK = NB>
__device__ void gfind(const Grp<GS>& q, const unsigned* h, int ra, int rb, CT& C, int& ba, int& ca, int& bb, int& cb)
{
    constexpr int PER = NBK / GS;   // 4 .. 32 consecutive buckets per thread, read as uint4
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
#pragma unroll
    for (int i = 0; i < GS / 32; ++i) base += i < w ? C.red[q.g][i] : 0;
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

// One scan of h[0..NB) by the group locating the buckets of NR ranks rk[] (each below the total): for
// each, the bucket, the keys below it and the keys in it.  With PREFIX, h becomes its inclusive prefix
// counts in the same pass.
template <int GS, int NR, bool PREFIX>
__device__ __forceinline__ void gfindn(const Grp<GS>& q, unsigned* h, const int (&rk)[NR], Ctl& C, int (&bo)[NR], int (&co)[NR],
                       int (&ho)[NR])
{
    constexpr int PER = NB / GS;
    const int lane = q.t & 31, w = q.t >> 5;
    int own = 0;
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
#pragma unroll
    for (int i = 0; i < GS / 32; ++i) base += i < w ? C.red[q.g][i] : 0;
    int c = base + incl - own;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int hk = (int)v[k];
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (c <= rk[j] && rk[j] < c + hk) {
                C.fr_b[q.g][j] = q.t * PER + k;
                C.fr_c[q.g][j] = c;
                C.fr_h[q.g][j] = hk;
            }
        }
        c += hk;
        if (PREFIX) v[k] = (unsigned)c;
    }
    if (PREFIX) {
#pragma unroll
        for (int k = 0; k < PER / 4; ++k) h4[k] = make_uint4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
    q.sync();
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        bo[j] = C.fr_b[q.g][j];
        co[j] = C.fr_c[q.g][j];
        ho[j] = C.fr_h[q.g][j];
    }
    q.sync();
}

// Values and point indices of the 0-based ranks s1 <= s2 among the pairs (buf, ib)[0..cnt), ordered by
// value and then by point index, by the group.  The indices of one buffer are distinct, so every rank
// names one pair and the choice among equal values never depends on the gather order.
template <int GS, class CT>
__device__ void gpick(const Grp<GS>& q, const float* buf, const int* ib, int cnt, int s1, int s2, CT& C, float& o1,
                      float& o2, int& i1, int& i2)
{
    // tpk adjacent threads (one warp) rank one pair, each against every tpk-th pair, and add their counts:
    // small sets are ranked in about cnt / tpk dependent steps.  Every thread of the group runs the same
    // number of outer iterations, so the shuffles see whole warps.
    const int tpk = cnt * 8 <= GS ? 8 : (cnt * 4 <= GS ? 4 : (cnt * 2 <= GS ? 2 : 1));
    const int sub = q.t & (tpk - 1);
    for (int t0 = 0; t0 < cnt; t0 += GS / tpk) {
        const int t = t0 + q.t / tpk;
        const bool live = t < cnt;
        int r = 0;
        float v = 0.f;
        int iv = 0;
        if (live) {
            v = buf[t];
            iv = ib[t];
#pragma unroll 4
            for (int s = sub; s < cnt; s += tpk) {
                const float w2 = buf[s];
                r += (w2 < v) | ((w2 == v) & (ib[s] < iv));
            }
        }
        for (int o = 1; o < tpk; o <<= 1) r += __shfl_xor_sync(0xFFFFFFFFu, r, o);
        if (live && sub == 0) {
            if (r == s1) {
                C.pv1[q.g] = v;
                C.pi1[q.g] = iv;
            }
            if (r == s2) {
                C.pv2[q.g] = v;
                C.pi2[q.g] = iv;
            }
        }
    }
    q.sync();
    o1 = C.pv1[q.g];
    o2 = C.pv2[q.g];
    i1 = C.pi1[q.g];
    i2 = C.pi2[q.g];
    q.sync();
}

// Ranks s1 <= s2 among the pairs (buf, ib)[0..cnt), every value in [lo, hi], ordered like gpick, for
// sets too large for its all-pairs ranking: a 256-bucket histogram of the values (h2, 256 counters),
// one warp's scan locates the buckets of the two ranks, their few pairs move to (tb, ti) and gpick ranks
// them there.  Buckets are monotone in the value, so the rank of a pair is the count in lower buckets
// plus its rank within its own bucket.
constexpr int NB2 = 256;
static_assert(NB2 + 2 * CAP1H == NB, "D_P runs in the histogram area: NB2 counters, then CAP1H values and CAP1H indices");
template <int GS, class CT, int TCAP = CAP>
__device__ void gpick_wide(const Grp<GS>& q, const float* buf, const int* ib, int cnt, int s1, int s2, float lo,
                           float hi, unsigned* h2, float* tb, int* ti, CT& C, float& o1, float& o2, int& i1,
                           int& i2)
{
    if (cnt <= 64 || !(lo < hi)) {
        gpick(q, buf, ib, cnt, s1, s2, C, o1, o2, i1, i2);
        return;
    }
    float scale = __fdiv_rn((float)NB2, __fsub_rn(hi, lo));
    if (!(scale <= FLT_MAX)) scale = FLT_MAX;
    for (int b = q.t; b < NB2; b += GS) h2[b] = 0u;
    if (q.t == 0) C.gn[q.g] = 0;
    q.sync();
    auto bk = [&](float v) {
        const int b = __float2int_rz(__fmul_rn(__fsub_rn(v, lo), scale));
        return b < 0 ? 0 : (b > NB2 - 1 ? NB2 - 1 : b);
    };
    for (int t = q.t; t < cnt; t += GS) atomicAdd(&h2[bk(buf[t])], 1u);
    q.sync();
    if (q.t < 32) {
        constexpr int PER2 = NB2 / 32;
        const int lane = q.t;
        unsigned v[PER2];
        int own = 0;
#pragma unroll
        for (int k = 0; k < PER2; ++k) {
            v[k] = h2[lane * PER2 + k];
            own += (int)v[k];
        }
        int incl = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        int c = incl - own;
#pragma unroll
        for (int k = 0; k < PER2; ++k) {
            const int hk = (int)v[k];
            if (hk > 0) {
                if (c <= s1 && s1 < c + hk) {
                    C.f_b1[q.g] = lane * PER2 + k;
                    C.f_c1[q.g] = c;
                }
                if (c <= s2 && s2 < c + hk) {
                    C.f_b2[q.g] = lane * PER2 + k;
                    C.f_c2[q.g] = c;
                }
            }
            c += hk;
        }
    }
    q.sync();
    const int b1 = C.f_b1[q.g], c1 = C.f_c1[q.g], b2 = C.f_b2[q.g];
    const int n2 = C.f_c2[q.g] + (int)h2[b2] - c1;
    if (n2 > TCAP) {   // the rank buckets hold more pairs than (tb, ti): rank the whole set
        gpick(q, buf, ib, cnt, s1, s2, C, o1, o2, i1, i2);
        return;
    }
    for (int t = q.t; t < cnt; t += GS) {
        const float v = buf[t];
        const int b = bk(v);
        if (b >= b1 && b <= b2) {
            const int pos = atomicAdd(&C.gn[q.g], 1);
            if (pos < TCAP) {
                tb[pos] = v;
                ti[pos] = ib[t];
            }
        }
    }
    q.sync();
    gpick(q, tb, ti, n2, s1 - c1, s2 - c1, C, o1, o2, i1, i2);
}

// Generic exact selection of ranks q1 <= q2 over one direction's values f(0..L-1),
// all in [lo, hi], by iterated bucketing (the fallback path); hist, buf and ibuf are the
// direction's own areas.  Returns the values and the point indices of the two ranks.
template <int GS, class CT, class F, int FBN = FB_NB, int FBC = FB_CAP>
__device__ void gselect(const Grp<GS>& q, F f, int L, int q1, int q2, float lo, float hi, unsigned* hist, float* buf,
                        int* ibuf, CT& C, float& v1, float& v2, int& i1, int& i2, int* err)
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
        float scale = __fdiv_rn((float)FBN, __fsub_rn(hi, lo));
        if (!(scale <= FLT_MAX)) scale = FLT_MAX;
        for (int b = q.t; b < FBN / 4; b += GS) reinterpret_cast<uint4*>(hist)[b] = make_uint4(0u, 0u, 0u, 0u);
        q.sync();
        for (int i = q.t; i < L; i += GS) {
            const float a = f(i);
            if (a >= lo && a <= hi) atomicAdd(&hist[bucket<FBN>(a, lo, scale)], 1u);
        }
        q.sync();
        int b1, c1, b2, c2;
        gfind<GS, CT, FBN>(q, hist, q1 - below, q2 - below, C, b1, c1, b2, c2);
        const int cnt = c2 + (int)hist[b2] - c1;
        if (q.t == 0) C.gn[q.g] = 0;
        q.sync();
        if (cnt <= FBC) {
            for (int i = q.t; i < L; i += GS) {
                const float a = f(i);
                if (a >= lo && a <= hi) {
                    const int b = bucket<FBN>(a, lo, scale);
                    if (b >= b1 && b <= b2) {
                        const int pos = atomicAdd(&C.gn[q.g], 1);
                        if (pos < FBC) {
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
                const int b = bucket<FBN>(a, lo, scale);
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

// Row i of X as D4 floats (D4 <= ldx, the padding zero): from the dataset's tiled copy Xt when it keeps
// one, else from the padded rows; the same values either way.  The projection pass streams X once per CTA
// and is bound by the cache lines its loads touch: a warp reading chunk c of 32 consecutive rows reads 512
// contiguous bytes of Xt, where in the padded rows the same 32 chunks lie on every line of the 32 rows.
template <int D4>
__device__ __forceinline__ void load_row(const DsDev& D, int i, int ldx, float (&xv)[D4])
{
    const float4* xr = D.Xt ? reinterpret_cast<const float4*>(D.Xt) + ((int64_t)(i >> 5) * (ldx >> 2)) * 32 + (i & 31)
                            : reinterpret_cast<const float4*>(D.X32 + (int64_t)i * ldx);
    const int cs = D.Xt ? 32 : 1;   // float4 stride between the chunks of one row
#pragma unroll
    for (int c = 0; c < D4 / 4; ++c) {
        const float4 t4 = xr[c * cs];
        xv[4 * c] = t4.x;
        xv[4 * c + 1] = t4.y;
        xv[4 * c + 2] = t4.z;
        xv[4 * c + 3] = t4.w;
    }
}

// Pass A of k_pdap2 for d <= 16 (D4 = d rounded up to 4, the directions uu in registers): the keys of G
// directions for the points i = tid + k NTK, stored (unless STREAM) and counted in the directions' histograms.
// xp points at row tid; CS is the float4 distance between the 16-byte chunks of one row (32 in the tiled
// copy Xt, 1 in the padded rows).  In both layouts rows i and i + NTK lie rstep = NTK ldx / 4 float4 apart
// (NTK is a multiple of 32, so i mod 32 stays put within a tile), so a thread walks its rows by a pointer
// increment and every chunk load takes a constant offset.  Two rows per iteration keep six loads in flight.
template <int G, int D4, bool STREAM, int CS, int NTK>
__device__ __forceinline__ void pass_a_rows(const float4* __restrict__ xp, size_t rstep, int tid, int n, int kst,
                                            const float (&uu)[G][D4], const float (&sc)[G], const float (&of)[G],
                                            float* keys, unsigned* hist)
{
    float* kq = keys + tid;   // key of direction g for the thread's current row: kq[g * kst]
    int i = tid;
    for (; i + NTK < n; i += 2 * NTK, xp += 2 * rstep, kq += 2 * NTK) {
        const float4* xq = xp + rstep;
        float xa[D4], xb[D4];
#pragma unroll
        for (int c = 0; c < D4 / 4; ++c) {
            const float4 a = xp[c * CS], b = xq[c * CS];
            xa[4 * c] = a.x;
            xa[4 * c + 1] = a.y;
            xa[4 * c + 2] = a.z;
            xa[4 * c + 3] = a.w;
            xb[4 * c] = b.x;
            xb[4 * c + 1] = b.y;
            xb[4 * c + 2] = b.z;
            xb[4 * c + 3] = b.w;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float ka = key_halves<D4>(uu[g], xa), kb = key_halves<D4>(uu[g], xb);
            if (!STREAM) {
                kq[g * kst] = ka;
                kq[g * kst + NTK] = kb;
            }
            atomicAdd(&hist[g * NB + bucket_m(ka, sc[g], of[g])], 1u);
            atomicAdd(&hist[g * NB + bucket_m(kb, sc[g], of[g])], 1u);
        }
    }
    if (i < n) {
        float xa[D4];
#pragma unroll
        for (int c = 0; c < D4 / 4; ++c) {
            const float4 a = xp[c * CS];
            xa[4 * c] = a.x;
            xa[4 * c + 1] = a.y;
            xa[4 * c + 2] = a.z;
            xa[4 * c + 3] = a.w;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float ka = key_halves<D4>(uu[g], xa);
            if (!STREAM) kq[g * kst] = ka;
            atomicAdd(&hist[g * NB + bucket_m(ka, sc[g], of[g])], 1u);
        }
    }
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

// D_P's MAD runs, found from the key histogram H of one direction before its median is known.  With the
// median run [ba, bb] (w buckets), let ss be the smallest s with more than k2 keys in the buckets
// [ba - s, bb + s]; the MAD ranks then deviate from the median by more than (ss - 2) and less than
// (ss + w) bucket widths, so their keys lie in two runs L, R at bucket distance about ss on either side.
// The runs taken here add two buckets on each side of that band, which lets the bound check of
// mad_from_runs pass; they are symmetric about (ba + bb) / 2: L = [L0, L1] below the median run and
// R = [R0, R1] above it.  H holds inclusive prefix counts (gfindn with PREFIX).  The runs stay unset (r untouched) when they would
// overlap the median run or the edge buckets, or hold more than cap keys.
template <int GS, class CT>
__device__ __forceinline__ void mad_runs(const Grp<GS>& q, unsigned* H, CT& C, int ba, int bb, int k2, int cap, int4& r,
                         int& cnt1, int& c_in)
{
    if (q.t == 0) C.f_b1[q.g] = NB;
    q.sync();
    // the window count is non-decreasing in s: rounds of GS consecutive values of s, one per thread, so
    // consecutive threads read consecutive prefix counts (no bank conflicts), until one exceeds k2; it
    // does by s = NB - 1, where the window holds all n keys
    int ss = NB;
    for (int s0 = 0; s0 < NB; s0 += GS) {
        const int s = s0 + q.t;
        const int hi = bb + s < NB - 1 ? bb + s : NB - 1, lo = ba - s;
        const int c = (int)H[hi] - (lo >= 1 ? (int)H[lo - 1] : 0);
        if (c > k2) atomicMin(&C.f_b1[q.g], s);
        q.sync();
        ss = C.f_b1[q.g];
        q.sync();
        if (ss < NB) break;
    }
    const int w = bb - ba + 1;
    const int L0 = ba - ss - w - 2, L1 = ba - ss + w + 3, R0 = bb + ss - w - 3, R1 = bb + ss + w + 2;
    if (ss >= w + 4 && L0 >= 1 && R1 <= NB - 2) {
        const int cl = (int)(H[L1] - H[L0 - 1]) + (int)(H[R1] - H[R0 - 1]);
        if (cl <= cap) {
            cnt1 = cl;
            c_in = (int)(H[R0 - 1] - H[L1]);
            r = make_int4(L0, L1, R0, R1);
        }
    }
}

// D_P's MAD from the gathered runs L, R (keys B1[0..cnt1), point indices I1) once the median m is known:
// the deviations replace the keys in place and the ranks s1 <= s2 among them are picked (gpick_wide, with
// h2 and the TCAP pairs tb / ti as scratch).  Every key between the runs lies in (max L, min R) and every
// key outside them below min L or above max R, so the picks are the MAD ranks of all keys when the
// deviations those bounds allow do not cross them; returns whether they do not (else nothing is picked
// for sure and the caller takes the |y - med| histogram pass).
template <int GS, int TCAP, class CT>
__device__ bool mad_from_runs(const Grp<GS>& q, float* B1, int* I1, int cnt1, int s1, int s2, float m, unsigned* h2,
                              float* tb, int* ti, CT& C, float& p1, float& p2, int& ip1, int& ip2)
{
    float lmin = FLT_MAX, lmax = -FLT_MAX, rmin = FLT_MAX, rmax = -FLT_MAX;
    for (int t = q.t; t < cnt1; t += GS) {
        const float v = B1[t];
        if (v < m) {   // L keys lie below m1 <= m, R keys above m2 >= m
            lmin = fminf(lmin, v);
            lmax = fmaxf(lmax, v);
        } else {
            rmin = fminf(rmin, v);
            rmax = fmaxf(rmax, v);
        }
        B1[t] = fabsf(__fsub_rn(v, m));
    }
    gminmax2(q, lmin, lmax, rmin, rmax, C);
    const float la = lmin, lb = lmax, ra = rmin, rb = rmax;
    if (!(lb > -FLT_MAX && ra < FLT_MAX && s1 >= 0 && s2 < cnt1)) return false;
    const float inner = fmaxf(__fsub_rn(m, lb), __fsub_rn(ra, m));
    const float outer = fminf(__fsub_rn(m, la), __fsub_rn(rb, m));
    gpick_wide<GS, CT, TCAP>(q, B1, I1, cnt1, s1, s2, fminf(__fsub_rn(m, lb), __fsub_rn(ra, m)),
                             fmaxf(__fsub_rn(m, la), __fsub_rn(rb, m)), h2, tb, ti, C, p1, p2, ip1, ip2);
    return inner <= p1 && outer >= p2;
}

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

// The points a selection kernel picked for one direction are written into the direction's result cell in
// place of its depth, which k_pdap_finish then forms from them: the points of the median ranks (im1, im2)
// and of the MAD or MAD_+ ranks (ip1, ip2); -1 where a selection failed (its error flag is set), and
// ip1 = ip2 = NOPOS for D_AP when no key lies above the median (MAD_+ = 0).  Two 8-byte stores: a result
// cell is 8-byte aligned.
constexpr int NOPOS = -2;
__device__ __forceinline__ void put_picks(ResDev* cell, int im1, int im2, int ip1, int ip2)
{
    int2* c = reinterpret_cast<int2*>(cell);
    c[0] = make_int2(im1, im2);
    c[1] = make_int2(ip1, ip2);
}

// FP64 finish of a selection launch: the depth of every direction from its picks (put_picks).  Four
// threads per direction, one per picked point, each forming the point's FP64 projection (proj64: one
// sequential FMA chain over the dims, the order in which the direction generator forms y_z, so a query
// equal to a data point projects to the same value); the first of the four forms
//   D_P  = 1 / (1 + |y_z - med| / MAD),   D_AP = 1 / (1 + (y_z - med)_+ / MAD_+)      (Sec. 2)
// with med the mean of the two median points (even n: the mean of the middle pair, odd n: the point
// twice), and writes it over the picks.  A kernel of its own: with thousands of directions in flight the
// long FP64 latencies overlap, where inside a selection CTA they would hold up the whole group.
__global__ void __launch_bounds__(256) k_pdap_finish(const TaskDev* __restrict__ tasks, int ntasks, int group,
                                                     const SlotDev* __restrict__ slots,
                                                     const DsDev* __restrict__ dsets, const float* __restrict__ U,
                                                     const double* __restrict__ yz, ResDev* __restrict__ res)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = (int)(t & 3);
    const int64_t dir = t >> 2;
    const int64_t ti = dir / group;
    const int g = (int)(dir - ti * group);
    bool live = ti < ntasks;
    TaskDev T{};
    if (live) {
        T = tasks[ti];
        live = g < T.nj;
    }
    double y = 0.0;
    int2 a = make_int2(-1, -1), b = make_int2(-1, -1);
    bool ap = false;
    double yzv = 0.0;
    ResDev* cell = nullptr;
    if (live) {
        const SlotDev& S = slots[T.slot];
        const DsDev& D = dsets[T.ds];
        cell = res + S.roff + T.j0 + g;
        a = reinterpret_cast<const int2*>(cell)[0];
        b = reinterpret_cast<const int2*>(cell)[1];
        ap = S.kind == 2;
        yzv = yz[S.roff + T.j0 + g];
        const int sel = k == 0 ? a.x : (k == 1 ? a.y : (k == 2 ? b.x : b.y));
        if (sel >= 0) y = proj64(D, U + S.uoff + (int64_t)(T.j0 + g) * D.ldx, sel);
    }
    // every lane of the warp takes part in the shuffles; the four lanes of a direction are adjacent
    const int lane = threadIdx.x & 31, l0 = lane & ~3;
    const double y0 = __shfl_sync(0xFFFFFFFFu, y, l0), y1 = __shfl_sync(0xFFFFFFFFu, y, l0 + 1);
    const double y2 = __shfl_sync(0xFFFFFFFFu, y, l0 + 2), y3 = __shfl_sync(0xFFFFFFFFu, y, l0 + 3);
    if (!live || k != 0) return;
    const int im1 = a.x, im2 = a.y, ip1 = b.x, ip2 = b.y;
    double depth = __longlong_as_double(0x7FF8000000000000LL);   // a failed selection (error flag set)
    if (im1 >= 0 && im2 >= 0) {
        const double med = (y0 + y1) * 0.5;
        if (ap) {
            double madp = 0.0;
            if (ip1 != NOPOS) madp = ip1 >= 0 && ip2 >= 0 ? fmax(((y2 - med) + (y3 - med)) * 0.5, 0.0) : depth;
            depth = depth_from(yzv - med > 0.0 ? yzv - med : 0.0, madp);
        } else if (ip1 >= 0 && ip2 >= 0) {
            depth = depth_from(fabs(yzv - med), (fabs(y2 - med) + fabs(y3 - med)) * 0.5);
        }
    }
    *cell = ResDev{depth, -1};
}

// Exact median / MAD / MAD_+ of one direction's keys y (after the projection pass), by its group q of
// GS threads.  The selection runs on the FP32 keys and yields the points holding the wanted order
// statistics (ties broken by point index), written to the direction's result cell (put_picks);
// k_pdap_finish forms the depth from FP64 projections of those few points and the FP64 y_z.
//   median  the bucket run of ranks k1, k2 (from the key histogram H) is gathered and ranked;
//   D_P     a |y - med| histogram pass, then the gather and ranking of the MAD run;
//   D_AP    in the median's gather pass, the run of the MAD_+ ranks guessed for no key tying the median.
// Runs that overflow the gather buffer fall back to iterated bucket selection.
// The gather pass of select_dir: every key whose raw bucket value lies in the median run [ml, ml + wm]
// moves, with its point index, to (B0, I0); every key in one of the NR2 second runs [l1, l1 + w1],
// [l2, l2 + w2] to (B1, I1), which holds cap1 pairs (ranges of raw values, compared as unsigned
// differences).  Four keys are tested at once with no branch into a mask of eight bits (key k in the median
// run, in a second run); a thread then takes one pass per set bit, so a warp spends on the rare gathered keys
// only as many passes as its busiest thread.  The keys gathered, and so the picks, are those of a test key by
// key.
template <int GS, int NR2, class K>
__device__ __forceinline__ void gather_runs(const Grp<GS>& q, const K& y, int n, float sc, float of, int ml,
                                            unsigned wm, int l1, unsigned w1, int l2, unsigned w2, int* fill,
                                            float* B0, int* I0, float* B1, int* I1, int cap1)
{
    auto in0 = [&](int rv) { return (unsigned)rv - (unsigned)ml <= wm; };
    auto in1 = [&](int rv) {
        bool h = false;
        if (NR2 >= 1) h = (unsigned)rv - (unsigned)l1 <= w1;
        if (NR2 >= 2) h = h | ((unsigned)rv - (unsigned)l2 <= w2);
        return h;
    };
    // one gathered key: set 0 (the median run) or 1 (the second runs)
    auto put = [&](int set, float v, int i) {
        const int pos = atomicAdd(&fill[set], 1);
        if (pos < (set ? cap1 : CAP)) {
            (set ? B1 : B0)[pos] = v;
            (set ? I1 : I0)[pos] = i;
        }
    };
    const int n4 = n & ~3;
    for (int i = 4 * q.t; i < n4; i += 4 * GS) {
        const float4 y4 = y.get4(i);
        const int r0 = bucket_raw(y4.x, sc, of), r1 = bucket_raw(y4.y, sc, of), r2 = bucket_raw(y4.z, sc, of),
                  r3 = bucket_raw(y4.w, sc, of);
        // bit k: key k in the median run; bit 4 + k: key k in a second run
        unsigned mk = (unsigned)in0(r0) | ((unsigned)in0(r1) << 1) | ((unsigned)in0(r2) << 2) |
                      ((unsigned)in0(r3) << 3) | ((unsigned)in1(r0) << 4) | ((unsigned)in1(r1) << 5) |
                      ((unsigned)in1(r2) << 6) | ((unsigned)in1(r3) << 7);
        while (mk) {   // one pass per gathered key of this thread (most threads: none)
            const int b = __ffs(mk) - 1;
            mk &= mk - 1;
            const int k = b & 3;
            const float v = k == 0 ? y4.x : (k == 1 ? y4.y : (k == 2 ? y4.z : y4.w));
            put(b >> 2, v, i + k);
        }
    }
    for (int i = n4 + q.t; i < n; i += GS) {
        const float v = y.get(i);
        const int rv = bucket_raw(v, sc, of);
        if (in0(rv)) put(0, v, i);
        if (NR2 > 0 && in1(rv)) put(1, v, i);
    }
}

template <int GS, class K>
__device__ __forceinline__ void select_dir(const Grp<GS>& q, const K& y, Ctl& C, unsigned* H, float* B0, int* I0,
                                           int n, bool ap, const DsDev& D, int64_t roff, ResDev* __restrict__ res,
                                           int* err)
{
    const int g = q.g;
    float* B1 = B0 + CAP;   // CAP1 entries: MAD_+ guess run (D_AP) or the runs L, R / the MAD run (D_P)
    int* I1 = I0 + CAP;
    const float sc = C.sc_y[g], of = C.off_y[g];
    const int k1 = (n - 1) / 2, k2 = n / 2;
    const int n4 = n & ~3;
    const float qnan = __int_as_float(0x7FC00000);
    constexpr int OFF = 1 << 30;   // a run start no bucket test can reach

    // one histogram scan: the median ranks, and for D_AP the ranks of the MAD_+ run guessed for no key
    // tying the median (for D_P the scan leaves prefix counts for mad_runs)
    const int npos_guess = (n & 1) ? (n - 1) / 2 : n / 2;
    int ba, ca, bb, cb, hb;
    int b3 = 0, c3 = 0, b4 = 0, c4 = 0, h4 = 0;
    if (ap) {
        const int gb = n - npos_guess;
        const int rk[4] = {k1, k2, npos_guess > 0 ? gb + (npos_guess - 1) / 2 : k1,
                           npos_guess > 0 ? gb + npos_guess / 2 : k2};
        int bo[4], co[4], ho[4];
        gfindn<GS, 4, false>(q, H, rk, C, bo, co, ho);
        ba = bo[0], ca = co[0], bb = bo[1], cb = co[1], hb = ho[1];
        b3 = bo[2], c3 = co[2], b4 = bo[3], c4 = co[3], h4 = ho[3];
    } else {
        const int rk[2] = {k1, k2};
        int bo[2], co[2], ho[2];
        gfindn<GS, 2, true>(q, H, rk, C, bo, co, ho);
        ba = bo[0], ca = co[0], bb = bo[1], cb = co[1], hb = ho[1];
    }
    const int c_lo0 = ca, cnt0 = cb + hb - ca;
    int fb = cnt0 > CAP ? 1 : 0;   // 1: fall back for every statistic, 2: only for the spread
    // second gathered set: the buckets of one or two runs [r.x, r.y], [r.z, r.w] (x > y: no run)
    int4 r2 = make_int4(OFF, -OFF, OFF, -OFF);
    int c_lo1 = 0, cnt1 = 0, c_in = 0;
    if (ap && npos_guess > 0) {
        c_lo1 = c3;
        cnt1 = c4 + h4 - c3;
        if (cnt1 > CAP1) fb = 1;
        r2 = make_int4(b3, b4, OFF, -OFF);   // the run [b3, b4]
    } else if (!ap && !fb) {
        mad_runs(q, H, C, ba, bb, k2, CAP1H, r2, cnt1, c_in);
    }
    const bool second = r2.x <= r2.y;
    // D_P runs of more than CAP1 keys go to the histogram area past the NB2 counters of the MAD pick: H is
    // idle from mad_runs until mad_from_runs, which uses only those counters (the |y - med| pass, which
    // clears all of H, needs the runs no more)
    const bool runs_in_h = !ap && second && cnt1 > CAP1;
    float* R1 = runs_in_h ? reinterpret_cast<float*>(H + NB2) : B1;
    int* J1 = runs_in_h ? reinterpret_cast<int*>(H + NB2 + CAP1H) : I1;
    const int cap1 = runs_in_h ? CAP1H : CAP1;
    float m1 = qnan, m2 = qnan, p1 = 0.f, p2 = 0.f;
    int im1 = -1, im2 = -1, ip1 = -1, ip2 = -1;
    int npos = 0;
    if (!fb) {
        if (q.t < 2) C.fill[g][q.t] = 0;
        q.sync();
        // the runs as ranges of raw bucket values (the edge buckets take every value clamped into them)
        const int ml = raw_lo(ba);
        const unsigned wm = (unsigned)raw_hi(bb) - (unsigned)ml;
        const bool two_runs = second && r2.z <= r2.w;
        const int l1 = second ? raw_lo(r2.x) : 0, l2 = two_runs ? raw_lo(r2.z) : 0;
        const unsigned w1 = second ? (unsigned)raw_hi(r2.y) - (unsigned)l1 : 0u;
        const unsigned w2 = two_runs ? (unsigned)raw_hi(r2.w) - (unsigned)l2 : 0u;
        int* fill = &C.fill[g][0];
        if (two_runs)
            gather_runs<GS, 2>(q, y, n, sc, of, ml, wm, l1, w1, l2, w2, fill, B0, I0, R1, J1, cap1);
        else if (second)
            gather_runs<GS, 1>(q, y, n, sc, of, ml, wm, l1, w1, l2, w2, fill, B0, I0, R1, J1, cap1);
        else
            gather_runs<GS, 0>(q, y, n, sc, of, ml, wm, l1, w1, l2, w2, fill, B0, I0, R1, J1, cap1);
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
            if (!(second && mad_from_runs<GS, CAP>(q, R1, J1, cnt1, k1 - c_in, k2 - c_in, m, H, B0, I0, C, p1,
                                                       p2, ip1, ip2))) {
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
                    atomicAdd(&H[bucket_m(fabsf(__fsub_rn(y4.x, m)), scd, TWO23)], 1u);
                    atomicAdd(&H[bucket_m(fabsf(__fsub_rn(y4.y, m)), scd, TWO23)], 1u);
                    atomicAdd(&H[bucket_m(fabsf(__fsub_rn(y4.z, m)), scd, TWO23)], 1u);
                    atomicAdd(&H[bucket_m(fabsf(__fsub_rn(y4.w, m)), scd, TWO23)], 1u);
                }
                for (int i = n4 + q.t; i < n; i += GS)
                    atomicAdd(&H[bucket_m(fabsf(__fsub_rn(y.get(i), m)), scd, TWO23)], 1u);
                q.sync();
                int da, dca, db, dcb;
                gfind(q, H, k1, k2, C, da, dca, db, dcb);
                const int cntd = dcb + (int)H[db] - dca;
                if (cntd > CAP1) {
                    fb = 2;
                } else {
                    if (q.t == 0) C.fill[g][1] = 0;
                    q.sync();
                    const int bwd = db - da;
                    auto gd = [&](float v, int i) {
                        const float dv = fabsf(__fsub_rn(v, m));
                        const int b = bucket_m(dv, scd, TWO23);
                        if ((unsigned)(b - da) <= (unsigned)bwd) {
                            const int pos = atomicAdd(&C.fill[g][1], 1);
                            if (pos < CAP1) {
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

    // ---- the picks, for the FP64 finish (k_pdap_finish) ---------------------------------------
    if (q.t == 0) put_picks(res + roff + g, im1, im2, ap && npos == 0 ? NOPOS : ip1, ap && npos == 0 ? NOPOS : ip2);
}

// Every live direction of the CTA: group g of cta_threads<G>() / G threads handles direction g alone,
// on its keys in shared memory or (STREAM) on keys formed by launch_pdap_keys in global memory (kin), else
// on keys recomputed from X.
template <int G, int DP4, bool STREAM>
__device__ __forceinline__ void select_dirs(Ctl& C, const float* keys, const float* uS, unsigned* hist, float* buf,
                                            int* ibuf, int n, int npad, int kst, bool ap, const DsDev& D, int GA,
                                            int64_t roff, ResDev* __restrict__ res, int* err, const float* kin)
{
    constexpr int GS = cta_threads<G>() / G;   // threads per direction group
    const int tid = threadIdx.x;
    const Grp<GS> q{tid / GS, tid % GS};
    const int g = q.g;
    if (g >= GA) return;   // inert direction (no CTA-wide barrier follows)
    unsigned* H = hist + g * NB;
    float* B0 = buf + (size_t)g * (CAP + CAP1);   // two gather runs, contiguous (FB_CAP for the fallback)
    int* I0 = ibuf + (size_t)g * (CAP + CAP1);    // the point index of every gathered key
    const float* u = uS + (size_t)g * D.ldx;
    if (STREAM && kin) {
        const KeysArray y{kin + ((size_t)blockIdx.x * G + g) * npad};
        select_dir<GS>(q, y, C, H, B0, I0, n, ap, D, roff, res, err);
    } else if (STREAM) {
        const KeysRecomputed<DP4> y{D.X32, u, D.ldx, DP4 ? DP4 : ((D.d + 3) & ~3)};
        select_dir<GS>(q, y, C, H, B0, I0, n, ap, D, roff, res, err);
    } else {
        const KeysArray y{keys + (size_t)g * kst};
        select_dir<GS>(q, y, C, H, B0, I0, n, ap, D, roff, res, err);
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
                                                 ResDev* __restrict__ res, int* err, const float* __restrict__ kin)
{
    extern __shared__ __align__(128) float sm[];
    __shared__ Ctl C;
    const TaskDev T = tasks[blockIdx.x];
    const SlotDev& S = slots[T.slot];
    const DsDev D = dsets[T.ds];   // the task carries its dataset row, so both loads go out together
    const int n = (int)D.n, ldx = D.ldx, d = D.d, dp4 = DP4 ? DP4 : ((d + 3) & ~3);
    const bool ap = (S.kind == 2);
    const int tid = threadIdx.x;
    const int npad = (n + 3) & ~3;   // key stride of the keys formed by launch_pdap_keys (kin)
    // key stride in shared memory: a multiple of 32 floats, so every direction's keys start on a 128-byte
    // line and a warp's 32 consecutive keys take one shared-memory wavefront
    const int kst = pdap_key_stride(n);
    float* keys = sm;                                          // G x kst (none when STREAM)
    float* uS = keys + (STREAM ? (size_t)0 : (size_t)G * kst);   // G x ldx
    unsigned* hist = reinterpret_cast<unsigned*>(uS + (size_t)G * ldx);   // G x NB
    float* buf = reinterpret_cast<float*>(hist + (size_t)G * NB);        // G x (CAP + CAP1)
    int* ibuf = reinterpret_cast<int*>(buf + (size_t)G * (CAP + CAP1));  // G x (CAP + CAP1)

    const int GA = T.nj;   // live directions; groups GA..G-1 are inert
    constexpr int NTK = cta_threads<G>();
    for (int e = tid; e < G * ldx; e += NTK) uS[e] = (e / ldx < GA) ? U[S.uoff + (int64_t)T.j0 * ldx + e] : 0.0f;
    for (int e = tid; e < G * NB / 4; e += NTK) reinterpret_cast<uint4*>(hist)[e] = make_uint4(0u, 0u, 0u, 0u);
    // per-direction bucket range: the centre's projection +- 5 sigma_u (sigma_u^2 = u' Cov u),
    // or +- the radius about the centre when no covariance is kept.  Keys outside the range go
    // to the edge buckets, which keeps the bucket map monotone.  One warp per direction: lanes
    // take rows of Cov (the range is a heuristic, so its summation order is free); y_z keeps the
    // keys' own arithmetic (one lane, sequential FMAs).
    // The range warps read their direction from U itself (the values the CTA stages in uS), so the range
    // is formed while the staging goes on, before the one barrier.
    if ((tid >> 5) < G) {
        const int g = tid >> 5, lane = tid & 31;
        float yc = 0.0f, qf = 0.0f;
        if (g < GA && d <= 32) {
            // lane r holds u_r and forms (Cov u)_r from the other lanes' u_c: every load of the warp is
            // independent of the arithmetic, so they go out together
            const float* u = U + S.uoff + (int64_t)(T.j0 + g) * ldx;
            const float ur = lane < d ? u[lane] : 0.0f;
            if (lane < d) yc = __fmul_rn(ur, D.center[lane]);
            if (D.cov) {
                const float* crow = D.cov + lane * d;
                float w = 0.0f;
#pragma unroll 8
                for (int c = 0; c < d; ++c) {
                    const float uc = __shfl_sync(0xFFFFFFFFu, ur, c);
                    if (lane < d) w = fmaf(crow[c], uc, w);
                }
                qf = __fmul_rn(w, ur);
            }
        } else if (g < GA) {   // inert directions keep a zero direction, as staged
            const float* u = U + S.uoff + (int64_t)(T.j0 + g) * ldx;
            for (int r = lane; r < d; r += 32) yc = fmaf(u[r], D.center[r], yc);
            if (D.cov) {
                // lanes stride over the d x d entries, so the covariance loads are independent of each other
                for (int e = lane; e < d * d; e += 32) {
                    const int r = e / d, c2 = e - r * d;
                    qf = fmaf(D.cov[e], __fmul_rn(u[r], u[c2]), qf);
                }
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
            C.off_y[g] = __fadd_rn(__fmul_rn(-C.lo_b[g], C.sc_y[g]), TWO23);
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
                if (!STREAM) keys[(size_t)g * kst + i] = acc[g];
                atomicAdd(&hist[g * NB + bucket_m(acc[g], sc[g], of[g])], 1u);
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
                        if (!STREAM) keys[(size_t)g * kst + i + h] = kv[h];
                        atomicAdd(&hist[g * NB + bucket_m(kv[h], sc[g], of[g])], 1u);
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
                float xv[D4];
                load_row<D4>(D, i, ldx, xv);
                const float ka = key_halves<D4>(ua, xv), kb = key_halves<D4>(ub, xv);
                if (!STREAM) keys[(size_t)(2 * pair) * kst + i] = ka;
                atomicAdd(&hist[(2 * pair) * NB + bucket_m(ka, sca, ofa)], 1u);
                if (!STREAM) keys[(size_t)(2 * pair + 1) * kst + i] = kb;
                atomicAdd(&hist[(2 * pair + 1) * NB + bucket_m(kb, scb, ofb)], 1u);
            }
        } else if (DP4 > 0) {
            constexpr int D4 = DP4 > 0 ? DP4 : 4;
            float uu[G][D4];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int c = 0; c < D4 / 4; ++c) {
                    const float4 u4 = *reinterpret_cast<const float4*>(uS + g * ldx + 4 * c);
                    uu[g][4 * c] = u4.x;
                    uu[g][4 * c + 1] = u4.y;
                    uu[g][4 * c + 2] = u4.z;
                    uu[g][4 * c + 3] = u4.w;
                }
            const int c4 = ldx >> 2;
            const size_t rstep = (size_t)NTK * c4;
            if (D.Xt)
                pass_a_rows<G, D4, STREAM, 32, NTK>(reinterpret_cast<const float4*>(D.Xt) +
                                                        ((size_t)(tid >> 5) * c4 * 32 + (tid & 31)),
                                                    rstep, tid, n, kst, uu, sc, of, keys, hist);
            else
                pass_a_rows<G, D4, STREAM, 1, NTK>(reinterpret_cast<const float4*>(D.X32) + (size_t)tid * c4, rstep,
                                                   tid, n, kst, uu, sc, of, keys, hist);
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

    select_dirs<G, DP4, STREAM>(C, keys, uS, hist, buf, ibuf, n, npad, kst, ap, D, GA, S.roff + T.j0, res, err, kin);
}

// ---------------------------------------------------------------------------------------------
// Warp-per-direction selection, keys recomputed from X at every pass (d <= 16, n <= PDAPW_MAX_N)
// ---------------------------------------------------------------------------------------------
// One CTA of WPC warps takes up to WPC directions of one query; warp w owns direction w.  No key is
// stored: pass A (the whole CTA, one X row per thread, every direction) forms each key and counts it
// in its direction's histogram (16-bit counters, two per word); each warp then finds its runs (the
// median run and, in the same pass, the D_P MAD runs or the D_AP MAD_+ run, as in select_dir); the
// gather pass (the whole CTA again) re-forms every key with the same arithmetic and moves the keys of
// the runs, with their point indices, into the warps' buffers; each warp ranks its buffers and forms
// the depth from FP64 projections of the selected points.  X is read twice per WPC directions, the
// selection work of a direction stays inside its warp (no block barrier), and the key arithmetic is
// that of the other selection kernels, so every kernel selects the same points.
constexpr int WPC = PDAPW_DIRS;    // directions (warps) per CTA
constexpr int WNB = 2048;          // buckets per direction (16-bit counters, WNB / 2 words)
constexpr int WCAP0 = 128;         // median-run buffer
constexpr int WCAP1 = 448;         // MAD_+ run or MAD L, R runs buffer
constexpr int WFBN = 1024;         // fallback histogram: 32-bit counters in the same WNB / 2 words
constexpr int WNT = WPC * 32;

struct CtlW {
    float lo_b[WPC], sc_y[WPC], off_y[WPC], scale[WPC];
    int red[WPC][2];
    float fred[WPC][2 * NWARP];
    int fill[WPC][2];
    int f_b1[WPC], f_c1[WPC], f_b2[WPC], f_c2[WPC];
    float pv1[WPC], pv2[WPC];
    int pi1[WPC], pi2[WPC];
    int gn[WPC], gi[WPC];
    // gather-pass tests of every direction: bucket map (sc, off), median run [bl0, bl0 + bw0], second set
    // |2b - c2| in [dl2, dl2 + dw2]
    float4 pa[WPC];
    int4 pb[WPC];
    // deviation passes of D_P directions: (med, bucket scale, run start or OFF (0 before the run is known), run width)
    float4 dv[WPC];
    int ndev;
};

// Key of a point for exactly D dims: the two half chains of key_halves<DP4> without their zero-padded
// terms (a zero product leaves a chain unchanged), so the values are those of the other kernels.
template <int D>
__device__ __forceinline__ float key_w(const float* u, const float* x)
{
    constexpr int DP4 = (D + 3) & ~3, H2 = DP4 / 2, E0 = D < H2 ? D : H2;
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int l = 0; l < E0; ++l) p0 = fmaf(u[l], x[l], p0);
#pragma unroll
    for (int l = H2; l < D; ++l) p1 = fmaf(u[l], x[l], p1);
    return __fadd_rn(p0, p1);
}

// The warp's histogram words are stored transposed: word v (of 1,024) at (v mod 32) * 32 + v / 32, so
// when lane l walks words 32 l .. 32 l + 31 (its range of buckets) the 32 lanes read 32 banks.
__device__ __forceinline__ int hidx(int v) { return ((v & 31) << 5) | (v >> 5); }
__device__ __forceinline__ void h16_add(unsigned* h, int b) { atomicAdd(&h[hidx(b >> 1)], 1u << ((b & 1) << 4)); }
__device__ __forceinline__ int h16_get(const unsigned* h, int b)
{
    return (int)((h[hidx(b >> 1)] >> ((b & 1) << 4)) & 0xFFFFu);
}

// Buckets holding ranks ra <= rb (both below the total) of a transposed warp histogram, and the counts
// below each, by one warp.  P16: 2,048 buckets of 16-bit counters (two per word), else 1,024 buckets of
// 32-bit counters.  Lane l owns words 32 l .. 32 l + 31.
template <bool P16>
__device__ void wfind(const unsigned* h, int ra, int rb, int& ba, int& ca, int& bb, int& cb)
{
    const int lane = threadIdx.x & 31;
    int own = 0;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
        const unsigned wd = h[(j << 5) | lane];
        own += P16 ? (int)((wd & 0xFFFFu) + (wd >> 16)) : (int)wd;
    }
    int incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    int c = incl - own, fa = -1, fca = 0, fb = -1, fcb = 0;
    const bool mine = (c <= rb && ra < c + own);   // only lanes whose range meets [ra, rb] walk it
    if (mine) {
#pragma unroll 1
        for (int j = 0; j < 32; ++j) {
            const unsigned wd = h[(j << 5) | lane];
#pragma unroll
            for (int hh = 0; hh < (P16 ? 2 : 1); ++hh) {
                const int hk = P16 ? (int)((wd >> (16 * hh)) & 0xFFFFu) : (int)wd;
                const int b = P16 ? lane * 64 + 2 * j + hh : lane * 32 + j;
                if (hk > 0) {
                    if (c <= ra && ra < c + hk) {
                        fa = b;
                        fca = c;
                    }
                    if (c <= rb && rb < c + hk) {
                        fb = b;
                        fcb = c;
                    }
                }
                c += hk;
            }
        }
    }
    const int la = __ffs(__ballot_sync(0xFFFFFFFFu, fa >= 0)) - 1, lb = __ffs(__ballot_sync(0xFFFFFFFFu, fb >= 0)) - 1;
    ba = __shfl_sync(0xFFFFFFFFu, fa, la);
    ca = __shfl_sync(0xFFFFFFFFu, fca, la);
    bb = __shfl_sync(0xFFFFFFFFu, fb, lb);
    cb = __shfl_sync(0xFFFFFFFFu, fcb, lb);
}

// Inclusive prefix counts of a transposed 16-bit warp histogram in place (every count, and n, below 2^16).
__device__ void wprefix(unsigned* h)
{
    const int lane = threadIdx.x & 31;
    int own = 0;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
        const unsigned wd = h[(j << 5) | lane];
        own += (int)((wd & 0xFFFFu) + (wd >> 16));
    }
    int incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    unsigned run = (unsigned)(incl - own);
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
        const unsigned wd = h[(j << 5) | lane];
        const unsigned lo = run + (wd & 0xFFFFu), hi = lo + (wd >> 16);
        run = hi;
        h[(j << 5) | lane] = lo | (hi << 16);
    }
    __syncwarp();
}

// Prefix count through bucket b (0 for b < 0) of a histogram turned into prefix counts by wprefix.
__device__ __forceinline__ int wP(const unsigned* h, int b) { return b < 0 ? 0 : h16_get(h, b); }

// One direction's keys re-formed from X (the gather-pass arithmetic), for the warp's fallback passes.
template <int D>
struct KeysW {
    const float* X;
    const float* u;
    int ldx;
    __device__ __forceinline__ float get(int i) const
    {
        constexpr int DP4 = (D + 3) & ~3;
        const float4* xr = reinterpret_cast<const float4*>(X + (int64_t)i * ldx);
        float xv[DP4], uv[DP4];
#pragma unroll
        for (int c = 0; c < DP4 / 4; ++c) {
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
        return key_w<D>(uv, xv);
    }
};

// Ranks s1 <= s2 of the pairs (buf, ib)[0..cnt): all-pairs ranking for small sets, else the value range
// and gpick_wide (h2: NB2 words, tb / ti: TCAP pairs of scratch).
template <int GS, int TCAP, class CT>
__device__ void gpick_auto(const Grp<GS>& q, const float* buf, const int* ib, int cnt, int s1, int s2, unsigned* h2,
                           float* tb, int* ti, CT& C, float& o1, float& o2, int& i1, int& i2)
{
    if (cnt <= 64) {
        gpick(q, buf, ib, cnt, s1, s2, C, o1, o2, i1, i2);
        return;
    }
    float lo = FLT_MAX, hi = -FLT_MAX;
    for (int t = q.t; t < cnt; t += GS) {
        lo = fminf(lo, buf[t]);
        hi = fmaxf(hi, buf[t]);
    }
    gminmax(q, lo, hi, C, lo, hi);
    gpick_wide<GS, CT, TCAP>(q, buf, ib, cnt, s1, s2, lo, hi, h2, tb, ti, C, o1, o2, i1, i2);
}

// The warp's last part: the iterated-bucket fallbacks over re-formed keys where a run overflowed its
// buffer (fb = 1: every statistic; fb = 2: the spread only), then the picks (as in select_dir).
template <int D>
__device__ void close_warp(const Grp<32>& q, const KeysW<D>& y, CtlW& C, unsigned* H, float* B0, int* I0, int n,
                           bool ap, int fb, float m1, float m2, int im1, int im2, float p1, float p2, int ip1, int ip2,
                           int npos, ResDev* __restrict__ out, int* err)
{
    const int k1 = (n - 1) / 2, k2 = n / 2;
    if (fb) {
        float kl = FLT_MAX, kh = -FLT_MAX;
        for (int i = q.t; i < n; i += 32) {
            const float v = y.get(i);
            kl = fminf(kl, v);
            kh = fmaxf(kh, v);
        }
        gminmax(q, kl, kh, C, kl, kh);
        auto f = [&](int i) { return y.get(i); };
        if (fb == 1)
            gselect<32, CtlW, decltype(f), WFBN, WCAP0 + WCAP1>(q, f, n, k1, k2, kl, kh, H, B0, I0, C, m1, m2, im1,
                                                                im2, err);
        if (ap) {
            int c = 0;
            for (int i = q.t; i < n; i += 32) c += (y.get(i) <= m1);
            const int nle = gsum(q, c, C);
            npos = n - nle;
            ip1 = ip2 = -1;
            if (npos > 0)
                gselect<32, CtlW, decltype(f), WFBN, WCAP0 + WCAP1>(q, f, n, nle + (npos - 1) / 2, nle + npos / 2, kl,
                                                                    kh, H, B0, I0, C, p1, p2, ip1, ip2, err);
        } else {
            const float m = __fmul_rn(__fadd_rn(m1, m2), 0.5f);
            const float dmax = fmaxf(fabsf(__fsub_rn(kl, m)), fabsf(__fsub_rn(kh, m)));
            auto fd = [&](int i) { return fabsf(__fsub_rn(y.get(i), m)); };
            gselect<32, CtlW, decltype(fd), WFBN, WCAP0 + WCAP1>(q, fd, n, k1, k2, 0.0f, dmax, H, B0, I0, C, p1, p2,
                                                                 ip1, ip2, err);
        }
    }
    if (q.t == 0) put_picks(out, im1, im2, ap && npos == 0 ? NOPOS : ip1, ap && npos == 0 ? NOPOS : ip2);
}

template <int D>
__global__ void __launch_bounds__(WNT, 2) k_pdapw(const TaskDev* __restrict__ tasks, const SlotDev* __restrict__ slots,
                                                   const DsDev* __restrict__ dsets, const float* __restrict__ U,
                                                   ResDev* __restrict__ res, int* err)
{
    constexpr int DP4 = (D + 3) & ~3;
    constexpr int OFF = 1 << 30;
    extern __shared__ __align__(16) float smw[];
    __shared__ CtlW C;
    const TaskDev T = tasks[blockIdx.x];
    const SlotDev& S = slots[T.slot];
    const DsDev Dd = dsets[S.ds];
    const int n = (int)Dd.n, ldx = Dd.ldx, d = Dd.d;
    const bool ap = (S.kind == 2);
    const int GA = T.nj;   // live directions; warps GA..WPC-1 are inert
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    float* uS = smw;                                                       // WPC x DP4
    unsigned* hist = reinterpret_cast<unsigned*>(uS + WPC * DP4);          // WPC x WNB / 2 words
    float* bufB = reinterpret_cast<float*>(hist + WPC * (WNB / 2));        // WPC x (WCAP0 + WCAP1)
    int* bufI = reinterpret_cast<int*>(bufB + WPC * (WCAP0 + WCAP1));      // WPC x (WCAP0 + WCAP1)
    for (int e = tid; e < WPC * DP4; e += WNT) {
        const int g = e / DP4, l = e - g * DP4;
        uS[e] = (g < GA && l < d) ? U[S.uoff + (int64_t)(T.j0 + g) * ldx + l] : 0.0f;
    }
    for (int e = tid; e < WPC * WNB / 8; e += WNT) reinterpret_cast<uint4*>(hist)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) C.ndev = 0;
    __syncthreads();
    // bucket range of direction w (as k_pdap2): the centre's projection +- 5 sigma_u, or +- the radius
    if (w < GA) {
        const float* u = uS + w * DP4;
        float yc = 0.0f, qf = 0.0f;
        for (int r = lane; r < d; r += 32) yc = fmaf(u[r], Dd.center[r], yc);
        if (Dd.cov) {
            for (int e = lane; e < d * d; e += 32) {
                const int r = e / d, c2 = e - r * d;
                qf = fmaf(Dd.cov[e], __fmul_rn(u[r], u[c2]), qf);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            yc += __shfl_xor_sync(0xFFFFFFFFu, yc, o);
            qf += __shfl_xor_sync(0xFFFFFFFFu, qf, o);
        }
        if (lane == 0) {
            float half = Dd.rc * 1.0001f;
            if (Dd.cov) {
                const float sg = sqrtf(fmaxf(qf, 0.0f));
                if (sg > 0.0f && 5.0f * sg < half) half = 5.0f * sg;
                C.scale[w] = sg;
            } else {
                C.scale[w] = half;
            }
            if (!(half > 0.0f)) half = fmaxf(fabsf(yc), 1.0f);
            C.lo_b[w] = yc - half;
            C.sc_y[w] = __fdiv_rn((float)WNB, __fadd_rn(half, half));
            C.off_y[w] = __fmul_rn(-C.lo_b[w], C.sc_y[w]);
        }
    }
    __syncthreads();

    // two rows per thread and iteration: the row loads of both are in flight together, and each direction's
    // vector is read from shared memory once for the two keys
    auto rows = [&](int i, float (&xa)[DP4], float (&xb)[DP4], bool two, int i2) {
        const float4* ra = reinterpret_cast<const float4*>(Dd.X32 + (int64_t)i * ldx);
        const float4* rb = reinterpret_cast<const float4*>(Dd.X32 + (int64_t)(two ? i2 : i) * ldx);
#pragma unroll
        for (int c = 0; c < DP4 / 4; ++c) {
            const float4 a = ra[c], b = rb[c];
            xa[4 * c] = a.x;
            xa[4 * c + 1] = a.y;
            xa[4 * c + 2] = a.z;
            xa[4 * c + 3] = a.w;
            xb[4 * c] = b.x;
            xb[4 * c + 1] = b.y;
            xb[4 * c + 2] = b.z;
            xb[4 * c + 3] = b.w;
        }
    };
    auto dir = [&](int g, float (&uu)[DP4]) {
#pragma unroll
        for (int c = 0; c < DP4 / 4; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(uS + g * DP4 + 4 * c);
            uu[4 * c] = v.x;
            uu[4 * c + 1] = v.y;
            uu[4 * c + 2] = v.z;
            uu[4 * c + 3] = v.w;
        }
    };

    // ---- pass A: every key of every direction counted in its histogram ------------------------
    for (int i = tid; i < n; i += 2 * WNT) {
        const int i2 = i + WNT;
        const bool two = i2 < n;
        float xa[DP4], xb[DP4];
        rows(i, xa, xb, two, i2);
#pragma unroll
        for (int g = 0; g < WPC; ++g) {
            if (g < GA) {
                float uu[DP4];
                dir(g, uu);
                const float sc = C.sc_y[g], of = C.off_y[g];
                unsigned* Hg = hist + g * (WNB / 2);
                h16_add(Hg, bucket_fma<WNB>(key_w<D>(uu, xa), sc, of));
                if (two) h16_add(Hg, bucket_fma<WNB>(key_w<D>(uu, xb), sc, of));
            }
        }
    }
    __syncthreads();

    // ---- each warp: the runs of its direction ---------------------------------------------------
    const int k1 = (n - 1) / 2, k2 = n / 2;
    unsigned* H = hist + w * (WNB / 2);
    int ba = 0, ca = 0, bb = 0, cb = 0, cnt0 = 0, c_lo1 = 0, cnt1 = 0, c_in = 0, fb = 0;
    bool lr_set = false;
    if (w < GA) {
        wfind<true>(H, k1, k2, ba, ca, bb, cb);
        cnt0 = cb + h16_get(H, bb) - ca;
        fb = cnt0 > WCAP0 ? 1 : 0;
        int c2 = 0, dl2 = OFF, dw2 = 0;
        const int npos_guess = (n & 1) ? (n - 1) / 2 : n / 2;
        if (ap && npos_guess > 0) {
            const int base = n - npos_guess;
            int b3, c3, b4, c4;
            wfind<true>(H, base + (npos_guess - 1) / 2, base + npos_guess / 2, b3, c3, b4, c4);
            c_lo1 = c3;
            cnt1 = c4 + h16_get(H, b4) - c3;
            if (cnt1 > WCAP1) fb = 1;
            c2 = 2 * b3 + (b4 - b3);
            dl2 = 0;
            dw2 = b4 - b3;
        } else if (!ap && !fb) {
            wprefix(H);
            // smallest s with more than k2 keys in the buckets [ba - s, bb + s] (the count grows with s and
            // reaches n at s = WNB - 1): 32 lanes at steps of 64, then 64 values two per lane
            auto win = [&](int s) {
                const int hi = bb + s < WNB - 1 ? bb + s : WNB - 1;
                return wP(H, hi) - wP(H, ba - s - 1);
            };
            const unsigned m1b = __ballot_sync(0xFFFFFFFFu, win(lane * 64) > k2);
            const int f1 = m1b ? __ffs(m1b) - 1 : 32;
            const int lo = f1 == 0 ? -1 : (f1 - 1) * 64;
            const int sa = lo + 1 + 2 * lane, sb = sa + 1;
            const unsigned ma = __ballot_sync(0xFFFFFFFFu, sa < WNB && win(sa) > k2);
            const unsigned mb = __ballot_sync(0xFFFFFFFFu, sb < WNB && win(sb) > k2);
            int ss = WNB;
            if (ma) ss = lo + 1 + 2 * (__ffs(ma) - 1);
            if (mb) ss = min(ss, lo + 2 + 2 * (__ffs(mb) - 1));
            // the runs L, R of mad_runs (two buckets beyond the band on each side)
            const int wd = bb - ba + 1;
            const int L0 = ba - ss - wd - 2, L1 = ba - ss + wd + 3, R0 = bb + ss - wd - 3, R1 = bb + ss + wd + 2;
            if (ss >= wd + 4 && L0 >= 1 && R1 <= WNB - 2) {
                const int cl = (wP(H, L1) - wP(H, L0 - 1)) + (wP(H, R1) - wP(H, R0 - 1));
                if (cl <= WCAP1) {
                    cnt1 = cl;
                    c_in = wP(H, R0 - 1) - wP(H, L1);
                    c2 = ba + bb;
                    dl2 = 2 * ss - wd - 7;
                    dw2 = 4 * wd + 10;
                    lr_set = true;
                }
            }
        }
        if (lane == 0) {
            C.pa[w] = make_float4(C.sc_y[w], C.off_y[w], __int_as_float(fb ? OFF : ba), __int_as_float(bb - ba));
            C.pb[w] = make_int4(c2, fb ? OFF : dl2, dw2, 0);
            C.fill[w][0] = 0;
            C.fill[w][1] = 0;
        }
    } else if (lane == 0) {
        C.pa[w] = make_float4(0.0f, 0.0f, __int_as_float(OFF), __int_as_float(0));
        C.pb[w] = make_int4(0, OFF, 0, 0);
    }
    __syncthreads();

    // ---- gather pass: the keys of every direction's runs, with their point indices ---------------
    for (int i = tid; i < n; i += 2 * WNT) {
        const int i2 = i + WNT;
        const bool two = i2 < n;
        float xa[DP4], xb[DP4];
        rows(i, xa, xb, two, i2);
#pragma unroll
        for (int g = 0; g < WPC; ++g) {
            if (g < GA) {
                float uu[DP4];
                dir(g, uu);
                const float4 pa = C.pa[g];
                const int4 pb = C.pb[g];
                const int bl0 = __float_as_int(pa.z), bw0 = __float_as_int(pa.w);
                float* Bg = bufB + g * (WCAP0 + WCAP1);
                int* Ig = bufI + g * (WCAP0 + WCAP1);
                auto put = [&](float v, int idx) {
                    const int b = bucket_fma<WNB>(v, pa.x, pa.y);
                    if ((unsigned)(b - bl0) <= (unsigned)bw0) {
                        const int pos = atomicAdd(&C.fill[g][0], 1);
                        if (pos < WCAP0) {
                            Bg[pos] = v;
                            Ig[pos] = idx;
                        }
                    }
                    if ((unsigned)(abs(2 * b - pb.x) - pb.y) <= (unsigned)pb.z) {
                        const int pos = atomicAdd(&C.fill[g][1], 1);
                        if (pos < WCAP1) {
                            Bg[WCAP0 + pos] = v;
                            Ig[WCAP0 + pos] = idx;
                        }
                    }
                };
                put(key_w<D>(uu, xa), i);
                if (two) put(key_w<D>(uu, xb), i2);
            }
        }
    }
    __syncthreads();

    // ---- each warp: ranks of its runs; D_P directions whose MAD runs did not hold (or overflowed) are
    // flagged for the deviation passes ------------------------------------------------------------
    const Grp<32> q{w, lane};
    const KeysW<D> y{Dd.X32, uS + w * DP4, ldx};
    float* B0 = bufB + w * (WCAP0 + WCAP1);
    int* I0 = bufI + w * (WCAP0 + WCAP1);
    float* B1 = B0 + WCAP0;
    int* I1 = I0 + WCAP0;
    float* tb = reinterpret_cast<float*>(H + NB2);   // pick scratch inside the histogram words
    int* ti = reinterpret_cast<int*>(H + NB2 + 256);
    constexpr int TC = 256;
    const float qnan = __int_as_float(0x7FC00000);
    float m1 = qnan, m2 = qnan, p1 = 0.f, p2 = 0.f, mf = 0.f, scd = 0.f;
    int im1 = -1, im2 = -1, ip1 = -1, ip2 = -1, npos = 0;
    bool dev = false;
    if (w < GA && !fb) {
        gpick_auto<32, TC>(q, B0, I0, cnt0, k1 - ca, k2 - ca, H, tb, ti, C, m1, m2, im1, im2);
        if (ap) {
            int c = 0;
            for (int t = lane; t < cnt0; t += 32) c += (B0[t] <= m1);
            const int nle = ca + gsum(q, c, C);
            npos = n - nle;
            if (npos > 0) {
                const int s3 = nle + (npos - 1) / 2 - c_lo1, s4 = nle + npos / 2 - c_lo1;
                if (s3 < 0 || s4 >= cnt1)
                    fb = 2;   // the positive count differed from the guess
                else
                    gpick_auto<32, TC>(q, B1, I1, cnt1, s3, s4, H, tb, ti, C, p1, p2, ip1, ip2);
            }
        } else {
            mf = __fmul_rn(__fadd_rn(m1, m2), 0.5f);
            const bool ok = lr_set && mad_from_runs<32, TC>(q, B1, I1, cnt1, k1 - c_in, k2 - c_in, mf, H, tb, ti, C,
                                                             p1, p2, ip1, ip2);
            if (!ok) {
                // |y - med| histogram over [0, 4 sigma_u] (edge bucket clamps) in the deviation passes
                float dmax = Dd.cov ? 4.0f * C.scale[w] : 0.0f;
                const float hard =
                    __fmul_rn(__fadd_rn(Dd.rc, fabsf(mf - C.lo_b[w] - 0.5f * (float)WNB / C.sc_y[w])), 1.0001f);
                if (!(dmax > 0.0f) || dmax > hard) dmax = hard;
                if (!(dmax > 0.0f)) dmax = 1.0f;
                scd = __fdiv_rn((float)WFBN, dmax);
                dev = true;
                for (int e = lane; e < WFBN; e += 32) H[e] = 0u;
            }
        }
    }
    if (lane == 0) {
        C.dv[w] = make_float4(mf, scd, __int_as_float(dev ? 0 : OFF), __int_as_float(0));
        if (dev) atomicAdd(&C.ndev, 1);
    }
    __syncthreads();

    if (C.ndev > 0) {
        // ---- deviation pass: |y - med| histograms of the flagged directions (32-bit, transposed) ----
        for (int i = tid; i < n; i += 2 * WNT) {
            const int i2 = i + WNT;
            const bool two = i2 < n;
            float xa[DP4], xb[DP4];
            rows(i, xa, xb, two, i2);
#pragma unroll 1
            for (int g = 0; g < GA; ++g) {
                const float4 dv = C.dv[g];
                if (__float_as_int(dv.z) != 0) continue;
                float uu[DP4];
                dir(g, uu);
                unsigned* Hg = hist + g * (WNB / 2);
                atomicAdd(&Hg[hidx(bucket_fma<WFBN>(fabsf(__fsub_rn(key_w<D>(uu, xa), dv.x)), dv.y, 0.0f))], 1u);
                if (two)
                    atomicAdd(&Hg[hidx(bucket_fma<WFBN>(fabsf(__fsub_rn(key_w<D>(uu, xb), dv.x)), dv.y, 0.0f))], 1u);
            }
        }
        __syncthreads();
        int da = 0, dca = 0, db = 0, dcb = 0, cntd = 0;
        if (dev) {
            wfind<false>(H, k1, k2, da, dca, db, dcb);
            cntd = dcb + (int)H[hidx(db)] - dca;
            if (cntd > WCAP1) {
                dev = false;
                fb = 2;
            }
            if (lane == 0) {
                C.dv[w].z = __int_as_float(dev ? da : OFF);
                C.dv[w].w = __int_as_float(db - da);
                C.fill[w][1] = 0;
            }
        }
        __syncthreads();
        // ---- deviation gather pass: the MAD runs of the flagged directions ----------------------------
        for (int i = tid; i < n; i += 2 * WNT) {
            const int i2 = i + WNT;
            const bool two = i2 < n;
            float xa[DP4], xb[DP4];
            rows(i, xa, xb, two, i2);
#pragma unroll 1
            for (int g = 0; g < GA; ++g) {
                const float4 dv = C.dv[g];
                const int lo = __float_as_int(dv.z), wdt = __float_as_int(dv.w);
                if (lo == OFF) continue;
                float uu[DP4];
                dir(g, uu);
                float* Bg = bufB + g * (WCAP0 + WCAP1) + WCAP0;
                int* Ig = bufI + g * (WCAP0 + WCAP1) + WCAP0;
                auto put = [&](float v, int idx) {
                    const float d1 = fabsf(__fsub_rn(v, dv.x));
                    if ((unsigned)(bucket_fma<WFBN>(d1, dv.y, 0.0f) - lo) <= (unsigned)wdt) {
                        const int pos = atomicAdd(&C.fill[g][1], 1);
                        if (pos < WCAP1) {
                            Bg[pos] = d1;
                            Ig[pos] = idx;
                        }
                    }
                };
                put(key_w<D>(uu, xa), i);
                if (two) put(key_w<D>(uu, xb), i2);
            }
        }
        __syncthreads();
        if (dev) gpick_auto<32, TC>(q, B1, I1, cntd, k1 - dca, k2 - dca, H, tb, ti, C, p1, p2, ip1, ip2);
    }

    if (w >= GA) return;   // no block barrier follows
    const int64_t ro = S.roff + T.j0 + w;
    close_warp<D>(q, y, C, H, B0, I0, n, ap, fb, m1, m2, im1, im2, p1, p2, ip1, ip2, npos, res + ro, err);
}

}  // namespace

size_t pdap_smem_bytes(int n, int group, int ldx, bool stream)
{
    const size_t kst = stream ? 0 : (size_t)pdap_key_stride(n);
    return sizeof(float) * ((size_t)group * kst + (size_t)group * ldx) + sizeof(unsigned) * (size_t)group * NB +
           (sizeof(float) + sizeof(int)) * (size_t)group * (CAP + CAP1);
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

int pdap_max_group(int n, int ldx, int m, int d, bool keys_in, bool allow_stream)
{
    // G in {1, 2, 4}: the largest G that fits two CTAs per SM when that is at least 2.  Below that the
    // keys go outside shared memory (0: formed once per round by a keys kernel, read at every pass),
    // which keeps four directions per SM in flight instead of one or two (measured on the 256-dataset
    // batched workload: the selection stage 8.2 s -> 5.4 s, identical results); callers that cannot
    // hold the keys elsewhere (allow_stream false) take the largest G that fits one CTA per SM.
    // Exception: for d > 16 with keys formed inside the kernel the projection pass re-reads X (4 d
    // bytes per point) for every G directions, so there the largest G that fits wins (measured at
    // n = 10,000: d = 50 1.27x, d = 150 1.68x faster with G = 4 than G = 2).
    const size_t one = pdap_smem_limit(), two = pdap_two_per_sm_limit();
    int g_one = 0, g_two = 0;
    for (int g = 1; g <= MAXG && g <= m; g *= 2) {
        const size_t need = pdap_smem_bytes(n, g, ldx);
        if (need <= one) g_one = g;
        if (need <= two) g_two = g;
    }
    if (pdap_dp4_class(d) == 0 && !keys_in) return g_one;
    if (g_two >= 2 || (g_two >= 1 && m < 2)) return g_two;
    return allow_stream ? 0 : g_one;
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

size_t pdapw_smem_bytes(int d)
{
    const size_t dp4 = (size_t)((d + 3) & ~3);
    return sizeof(float) * WPC * dp4 + sizeof(unsigned) * WPC * (WNB / 2) +
           (sizeof(float) + sizeof(int)) * WPC * (WCAP0 + WCAP1);
}

bool pdapw_eligible(int64_t n, int d) { return d >= 1 && d <= 16 && n >= 1 && n <= PDAPW_MAX_N; }

template <int D>
static cudaError_t launch_w(const TaskDev* tasks, int ntasks, const SlotDev* slots, const DsDev* ds, const float* U,
                            const double* yz, ResDev* res, int* err, cudaStream_t st)
{
    const size_t smem = pdapw_smem_bytes(D);
    cudaError_t e = cudaFuncSetAttribute(k_pdapw<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    k_pdapw<D><<<ntasks, WNT, smem, st>>>(tasks, slots, ds, U, res, err);
    return cudaGetLastError();
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
    k_pdap2<G, DP4, STREAM><<<ntasks, cta_threads<G>(), smem, st>>>(tasks, slots, ds, U, res, err, kin);
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

static cudaError_t launch_select(const TaskDev* tasks, int ntasks, size_t smem, int group, int variant,
                                 const SlotDev* slots, const DsDev* ds, const float* U, const double* yz, ResDev* res,
                                 int* err, cudaStream_t st, const float* kin);

cudaError_t launch_pdap(const TaskDev* tasks, int ntasks, size_t smem, int group, int variant, const SlotDev* slots,
                        const DsDev* ds, const float* U, const double* yz, ResDev* res, int* err, cudaStream_t st,
                        const float* kin)
{
    if (ntasks <= 0) return cudaSuccess;
    const cudaError_t e = launch_select(tasks, ntasks, smem, group, variant, slots, ds, U, yz, res, err, st, kin);
    if (e != cudaSuccess) return e;
    const int64_t threads = (int64_t)ntasks * group * 4;
    const int nt = 256;
    k_pdap_finish<<<(unsigned)((threads + nt - 1) / nt), nt, 0, st>>>(tasks, ntasks, group, slots, ds, U, yz, res);
    return cudaGetLastError();
}

static cudaError_t launch_select(const TaskDev* tasks, int ntasks, size_t smem, int group, int variant,
                                 const SlotDev* slots, const DsDev* ds, const float* U, const double* yz, ResDev* res,
                                 int* err, cudaStream_t st, const float* kin)
{
    if (smem > pdap_smem_limit()) return cudaErrorInvalidValue;
    if (variant & PDAP_WARP) {
        if (group < 1 || group > PDAPW_DIRS) return cudaErrorInvalidValue;
        switch (variant & 0xFF) {
        case 1: return launch_w<1>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 2: return launch_w<2>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 3: return launch_w<3>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 4: return launch_w<4>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 5: return launch_w<5>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 6: return launch_w<6>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 7: return launch_w<7>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 8: return launch_w<8>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 9: return launch_w<9>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 10: return launch_w<10>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 11: return launch_w<11>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 12: return launch_w<12>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 13: return launch_w<13>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 14: return launch_w<14>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 15: return launch_w<15>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        case 16: return launch_w<16>(tasks, ntasks, slots, ds, U, yz, res, err, st);
        default: return cudaErrorInvalidValue;
        }
    }
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
    if (group == PDAP_WARP_GROUP && pdapw_eligible(n, d)) {
        // one warp per direction, keys re-formed at every pass (taken when asked for: on the d = 10,
        // n = 10,000 workload it runs 1.2x slower than two directions per CTA with resident keys); the
        // query's m directions are spread evenly over its CTAs
        const int ctas = (m + PDAPW_DIRS - 1) / PDAPW_DIRS;
        s.group = (m + ctas - 1) / ctas;
        s.variant = PDAP_WARP | d;
        s.smem = pdapw_smem_bytes(d);
        s.keys_gemm = false;
        return s;
    }
    int G = (group == PDAP_WARP_GROUP || group == PDAP_STREAM_CHOICE) ? 0 : group;
    if (G && (G > m || pdap_smem_bytes(n, G, ldx) > pdap_smem_limit())) G = 0;
    if (!G && group != PDAP_STREAM_CHOICE) G = pdap_max_group(n, ldx, m, d, dp4 == 0, true);
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
