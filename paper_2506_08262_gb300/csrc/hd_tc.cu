// Halfspace depth counts on the tcgen05 tensor cores (Sec. 2, D_H; the projection
// Y = U X^T of Sec. 4.1 as a GEMM) with split-BF16x3 products.
//
// Every x and u is split into BF16 parts, x = x_hi + x_lo (+ residual), and
// u'x is formed as u_hi'x_hi + u_lo'x_hi + u_hi'x_lo with FP32 accumulation in
// tensor memory.  The query's projection is folded into the same GEMM: the
// data planes carry 1 in two spare K columns and the direction planes carry
// the BF16 parts of -u'z there, so the accumulator holds t = u'x - u'z
// directly.  The epilogue counts t < -b and t > b, b = gamma (|x| + |z|) a
// bound on the error of t; every |t| <= b is settled by a compensated FP32
// dot product (about twice FP32 precision) and, when even that is too close
// to call, by the exact FP64 sign test, so the counts are exact.
//
// CTA layout (640 threads): warp 0 streams point tiles with TMA into a
// 2-stage ring, warp 1 owns tensor memory and issues the MMAs, warps 2-17 read
// the accumulator (one accumulator row per TMEM lane, four warps per lane
// quarter, each taking one 32-column chunk of every tile) and count, and
// warps 18-19 settle near ties handed to them by the counting warps.  The 128
// rows of a CTA are consecutive (query, direction) pairs of one request, so
// one tile may hold several queries.  Tiles are 256 points wide for a K
// extent of 64 (four accumulator buffers of 128 columns otherwise); two
// 256-column accumulator buffers let the MMAs of one tile overlap the
// epilogue of the previous one.  Per chunk the epilogue packs
// the sign bits of t and of (b - |t|) into bit words (three instructions per
// column); columns inside the band go to a per-warp queue.  Each full batch
// of 32 is handed to the settle warps through a small ring in shared memory
// (settled inline when every slot is taken), so the slow test, one candidate
// per lane, stays off the path that frees the accumulator buffers.
// Every wait on an mbarrier is bounded; on timeout the CTA flags ERR_TIMEOUT
// and winds down.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "async_sync.cuh"
#include "rrs_device.cuh"
#include "rrs_internal.h"

namespace rrs {

namespace {

using namespace async;

constexpr int BM = 128;          // directions per CTA (TMEM lanes)
// Points per tile (accumulator columns, the MMA's N) is a template parameter: 256 when the
// K extent is 64 (a 128 x 256 x 16 MMA runs at the full tensor rate; 128 x 128 x 16 does
// not), 128 when it is 128 (two 256-point stages would not fit in shared memory).
constexpr int STAGES = 4;                    // largest TMA ring
constexpr int MAXACC = 4;                    // accumulator buffers: 512 TMEM columns / BN
constexpr int QCAP = 64;                     // near-tie queue entries per epilogue warp
constexpr int NEPI = 16;                     // epilogue warps: four per TMEM lane quarter
constexpr int NSET = 2;                      // settle warps
constexpr int NSLOT = 8;                     // batches of 32 near ties in flight to the settle warps
constexpr int NTHREADS = 64 + 32 * (NEPI + NSET);

__host__ __device__ constexpr int plane_bytes_rows(int rows) { return rows * 128; }   // one 64-wide K chunk

// instruction descriptor of tcgen05.mma kind::f16: BF16 A and B, FP32 accumulator,
// both operands K-major, M = 128, N = bn
__host__ __device__ constexpr uint32_t mma_idesc(int bn)
{
    return (1u << 4)                     // D format: FP32
           | (1u << 7)                   // A format: BF16
           | (1u << 10)                  // B format: BF16
           | ((uint32_t)(bn >> 3) << 17)
           | ((uint32_t)(BM >> 4) << 24);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of 1024 bytes
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // layout: 128-byte swizzle
    return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes (one row per thread);
// the registers are valid only after tmem_wait_ld / tmem_order
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
// wait for this thread's outstanding tcgen05.ld; the registers are in-out operands so no
// use of them can be scheduled before the wait
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]) : : "memory");
}
// byte offset of element (row, k) in a K chunk of 64 BF16 per row, 128-byte swizzle
__device__ __forceinline__ uint32_t sw128_offset(int row, int k)
{
    const int unit = (k >> 3) ^ (row & 7);
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + unit * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float bf16_val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

struct TcShared {
    uint64_t full[STAGES], acc_full[MAXACC], acc_empty[MAXACC];
    uint32_t tmem_base;
    int abort;
    int mma_tiles;   // tiles whose operands the MMA issuer has consumed
    unsigned zmax_bits;
    int sq_state[NSLOT];   // settle ring slots: SQ_FREE, SQ_FILLING, SQ_FULL, SQ_SETTLING
    int epi_done;          // counting warps that have handed off their last batch
};
enum { SQ_FREE = 0, SQ_FILLING = 1, SQ_FULL = 2, SQ_SETTLING = 3 };

// One accumulator row of the CTA: a (query, direction) pair.
struct RowInfo {
    long long uoff;   // element offset of the direction's FP32 row in U
    int roff;         // index of (query, direction) in y_z and in the results
    int zoff64;       // offset of the query's FP64 row
    float zn;         // |z|, rounded up
    float yh, yl;     // y_z = u'z as an unevaluated FP32 pair (|y_z - yh - yl| <= 2^-48 |y_z|)
    int slot;         // query slot (index of the near-tie counter)
};

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// Sign of t = u'x - y_z from a compensated FP32 dot product (error-free products and
// sums, errors gathered in a second float), i.e. t to about twice FP32 precision.
// Returns +1 / -1, or 0 when |t| does not clear twice the bound and the caller must
// take the exact test.  u and x are ldx-long rows (zero padded, 16-byte aligned).
__device__ __noinline__ int ff_sign(const float* __restrict__ u, const float* __restrict__ x, int ldx, float yh,
                                    float yl, float bound)
{
    float s = 0.f, c = 0.f;
    auto acc = [&](float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = __fmaf_rn(a, b, -p);   // exact: a b = p + pe
        float s2, se;
        two_sum_f(s, p, s2, se);
        s = s2;
        c = __fadd_rn(c, __fadd_rn(se, pe));
    };
    for (int l = 0; l < ldx; l += 4) {
        const float4 a = *reinterpret_cast<const float4*>(u + l);
        const float4 b = *reinterpret_cast<const float4*>(x + l);
        acc(a.x, b.x);
        acc(a.y, b.y);
        acc(a.z, b.z);
        acc(a.w, b.w);
    }
    float a, ea;
    two_sum_f(s, -yh, a, ea);
    const float t = __fadd_rn(a, __fadd_rn(ea, __fsub_rn(c, yl)));
    const float b2 = __fmul_rn(2.0f, bound);
    if (t > b2) return 1;
    if (t < -b2) return -1;
    return 0;
}

template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_hd_tc(const CUtensorMap* __restrict__ maps, const TaskDev* __restrict__ tasks,
            const SlotDev* __restrict__ slots, const DsDev* __restrict__ dsets, const float* __restrict__ U,
            const double* __restrict__ yz, const double* __restrict__ z64, ResDev* __restrict__ res,
            int64_t* __restrict__ band_out, int* err, float gamma, int nst)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ TcShared sh;
    __shared__ RowInfo rows[BM];
    constexpr int NACC = 512 / BN;                            // accumulator buffers
    constexpr int CPW = BN / 128;                             // 32-column chunks per epilogue warp and tile
    __shared__ __align__(16) float bcol[NEPI][32 * CPW];      // per-column band bound of the warp's chunks
    __shared__ uint32_t qpt[NEPI][QCAP];                      // candidate queue: point index
    __shared__ uint8_t qrow[NEPI][QCAP];                      //                  accumulator row
    __shared__ uint32_t sq_pt[NSLOT][32];                     // settle ring: point index
    __shared__ uint8_t sq_row[NSLOT][32];                     //              accumulator row
    __shared__ int cand_lt[BM], cand_gt[BM];                  // exact verdicts on candidates, per row
    __shared__ uint32_t partial_lt[NEPI][32], partial_gt[NEPI][32];

    if (*(volatile const int*)err & ERR_TIMEOUT) return;   // another CTA already gave up
    const TaskDev T = tasks[blockIdx.x];
    const int dsi = slots[T.slot].ds;
    const DsDev D = dsets[dsi];
    // the tensor map of this task's dataset (one per dataset in device memory, so one launch serves the
    // tasks of every dataset with the same K extent)
    const CUtensorMap* xmap = maps + dsi;
    const int kp = D.kp, nchunk = kp / 64, d = D.d, ldx = D.ldx;
    const float ffcoef = band_coef_ff(d);
    const int64_t n = D.n;
    const int ntiles = (int)((n + BN - 1) / BN);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // ---- rows: T covers rows j0 .. j0+nj-1 of its request's (query, direction) sequence,
    //      m directions per query, starting at query slot T.slot -------------------------
    if (threadIdx.x == 0) {
        sh.zmax_bits = 0u;
        for (int i = 0; i < NSLOT; ++i) sh.sq_state[i] = SQ_FREE;
        sh.epi_done = 0;
    }
    __syncthreads();
    if (threadIdx.x < BM) {
        const int r = threadIdx.x;
        RowInfo ri{};
        if (r < T.nj) {
            const int m = slots[T.slot].m;
            const int gg = T.j0 + r;
            const int qs = gg / m, j = gg - qs * m;
            const SlotDev& S = slots[T.slot + qs];
            ri.uoff = S.uoff + (long long)j * S.ldx;
            ri.roff = S.roff + j;
            ri.zoff64 = S.zoff64;
            ri.zn = S.znorm;
            ri.slot = T.slot + qs;
            const double y = yz[ri.roff];
            ri.yh = (float)y;
            ri.yl = (float)(y - (double)ri.yh);
            atomicMax(&sh.zmax_bits, __float_as_uint(S.znorm));
        }
        rows[r] = ri;
        cand_lt[r] = 0;
        cand_gt[r] = 0;
    }
    __syncthreads();

    // 1024-byte aligned operand area: A planes (hi, lo) then STAGES x B planes (hi, lo)
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t a_plane = (uint32_t)nchunk * plane_bytes_rows(BM);      // bytes of one A plane
    const uint32_t b_plane = (uint32_t)nchunk * plane_bytes_rows(BN);      // bytes of one B plane
    uint8_t* Ahi = base;
    uint8_t* Alo = base + a_plane;
    uint8_t* Bst = base + 2 * a_plane;                                     // stage s at Bst + s * 2 * b_plane

    // ---- A planes from the FP32 directions, with the folded -y_z columns ----------------
    for (int e = threadIdx.x; e < BM * kp; e += NTHREADS) {
        const int r = e / kp, k = e - r * kp;
        float hi = 0.f, lo = 0.f;
        if (r < T.nj) {
            if (k < d) {
                const float u = U[rows[r].uoff + k];
                hi = bf16_val(bf16_bits(u));
                lo = u - hi;   // exact in FP32
            } else if (k == d || k == d + 1) {
                const double y = yz[rows[r].roff];
                const float y1 = bf16_val(bf16_bits((float)y));
                const double r1 = y - (double)y1;
                const float y2 = bf16_val(bf16_bits((float)r1));
                const double r2 = r1 - (double)y2;
                const float y3 = bf16_val(bf16_bits((float)r2));
                if (k == d) {
                    hi = -y1;
                    lo = -y2;
                } else {
                    hi = 0.f;
                    lo = -y3;
                }
            }
        }
        const int c = k >> 6, kk = k & 63;
        const uint32_t off = (uint32_t)c * plane_bytes_rows(BM) + sw128_offset(r, kk);
        *reinterpret_cast<uint16_t*>(Ahi + off) = bf16_bits(hi);
        *reinterpret_cast<uint16_t*>(Alo + off) = bf16_bits(lo);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&sh.full[s], 1);
        }
        sh.mma_tiles = 0;
        for (int b = 0; b < NACC; ++b) {
            mbar_init(&sh.acc_full[b], 1);
            mbar_init(&sh.acc_empty[b], NEPI);   // one arrival per epilogue warp
        }
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                     "r"(NACC * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem_base;

    // exact verdicts on near ties: lane k of the calling warp takes entry k of (pts, rws)
    const double* X64 = D.X64;
    auto settle = [&](const uint32_t* pts, const uint8_t* rws, int cnt) {
        __syncwarp();
        if (lane < cnt) {
            const int64_t i = pts[lane];
            const int r = rws[lane];
            const RowInfo& R = rows[r];
            const float* ur = U + R.uoff;
            int sgn;
            if (X64) {
                sgn = rrsdev::exact_sign<double>(ur, 1, X64 + i * d, z64 + R.zoff64, d, err);
            } else {
                const float* xr = D.X32 + i * ldx;
                const float bnd = ffcoef * (D.xnorm[i] + R.zn) + (float)(d + 2) * 0x1p-140f;
                sgn = ff_sign(ur, xr, ldx, R.yh, R.yl, bnd);
                if (sgn == 0) sgn = rrsdev::exact_sign<float>(ur, 1, xr, z64 + R.zoff64, d, err);
            }
            if (sgn < 0) atomicAdd(&cand_lt[r], 1);
            else if (sgn > 0) atomicAdd(&cand_gt[r], 1);
            if (band_out) atomicAdd((unsigned long long*)&band_out[R.slot], 1ull);
        }
        __syncwarp();
    };

    if (warp == 0) {
        // ---- TMA producer ------------------------------------------------------------------
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)xmap) : "memory");
            int issued = 0;
            for (int t = 0; t < ntiles; ++t) {
                const int s = t % nst;
                // stage s is free once the MMAs of tile t - nst have completed, which the accumulator's
                // full barrier of that tile reports (one commit per tile serves both)
                const int u = t - nst;
                if (t >= nst && !mbar_wait(&sh.acc_full[u % NACC], (u / NACC) & 1, err)) {
                    atomicOr(err, ERR_TIMEOUT);
                    sh.abort = 1;
                    break;
                }
                if (*(volatile int*)&sh.abort) break;
                uint8_t* st = Bst + (size_t)s * 2 * b_plane;
                mbar_arrive_expect_tx(&sh.full[s], 2 * b_plane);
                for (int p = 0; p < 2; ++p)
                    for (int c = 0; c < nchunk; ++c)
                        tma_load_2d(st + p * b_plane + c * plane_bytes_rows(BN), xmap, p * kp + c * 64, t * BN,
                                    &sh.full[s]);
                issued = t + 1;
            }
            if (*(volatile int*)&sh.abort) {
                // do not leave copies in flight into this CTA's shared memory: wait (bounded) for the
                // loads the MMA issuer has not consumed
                for (int t = *(volatile int*)&sh.mma_tiles; t < issued; ++t) mbar_wait(&sh.full[t % nst], (t / nst) & 1, err, false);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ---------------------------------------------------------------------
        if (lane == 0) {
            const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo);
            for (int t = 0; t < ntiles; ++t) {
                const int s = t % nst, b = t % NACC;
                if (!mbar_wait(&sh.full[s], (t / nst) & 1, err) ||
                    (t >= NACC && !mbar_wait(&sh.acc_empty[b], ((t / NACC) - 1) & 1, err))) {
                    atomicOr(err, ERR_TIMEOUT);
                    sh.abort = 1;
                    break;
                }
                if (*(volatile int*)&sh.abort) break;
                tc_fence_after();
                const uint32_t bst = smem_u32(Bst + (size_t)s * 2 * b_plane);
                const uint32_t bhi = bst, blo = bst + b_plane;
                const uint32_t dtm = tmem + (uint32_t)(b * BN);
                uint32_t acc = 0;
                // products (A plane, B plane): (hi, hi), (lo, hi), (hi, lo)
                for (int pr = 0; pr < 3; ++pr) {
                    const uint32_t ap = pr == 1 ? alo : ahi;
                    const uint32_t bp = pr == 2 ? blo : bhi;
                    for (int c = 0; c < nchunk; ++c) {
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = sw128_desc(ap + c * plane_bytes_rows(BM) + ks * 32);
                            const uint64_t bd = sw128_desc(bp + c * plane_bytes_rows(BN) + ks * 32);
                            umma_bf16(dtm, ad, bd, mma_idesc(BN), acc);
                            acc = 1;
                        }
                    }
                }
                umma_commit(&sh.acc_full[b]);
                *(volatile int*)&sh.mma_tiles = t + 1;
            }
            const int done = *(volatile int*)&sh.mma_tiles;
            if (*(volatile int*)&sh.abort && done > 0) {
                // let the last issued MMAs finish before tensor memory is released
                const int t = done - 1;
                mbar_wait(&sh.acc_full[t % NACC], (t / NACC) & 1, err, false);
            }
        }
    } else if (warp < 2 + NEPI) {
        // ---- epilogue: one accumulator row (direction) per thread ---------------------------
        // Four warps share each TMEM lane quarter; warp e takes the 32-column chunk e / 4 of
        // every tile.  Per column the sign bits of t and of (bound - |t|) are shifted into bit
        // words (one add and two funnel shifts); the few columns inside the band go to a
        // per-warp queue whose batches of 32 go to the settle warps.
        const int e = warp - 2;                 // 0..NEPI-1
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int cw = e >> 2;                  // column chunk of each tile
        const int row = q * 32 + lane;          // accumulator row = TMEM lane
        const bool live = row < T.nj;
        const float gz = gamma * __uint_as_float(sh.zmax_bits);
        uint32_t lt = 0, gt = 0;                // n < 2^31
        int qn = 0;                             // queue fill (warp-uniform)

        // hand queue entries [b0, b0 + 32) to a free slot of the settle ring, or settle them here
        auto hand_off = [&](int b0) {
            __syncwarp();   // the entries were appended by several lanes
            int s = -1;
            if (lane == 0) {
                for (int k = 0; k < NSLOT; ++k) {
                    const int i = (e + k) & (NSLOT - 1);
                    if (*(volatile int*)&sh.sq_state[i] == SQ_FREE &&
                        atomicCAS(&sh.sq_state[i], SQ_FREE, SQ_FILLING) == SQ_FREE) {
                        s = i;
                        break;
                    }
                }
            }
            s = __shfl_sync(0xFFFFFFFFu, s, 0);
            if (s < 0) {
                settle(&qpt[e][b0], &qrow[e][b0], 32);
                return;
            }
            sq_pt[s][lane] = qpt[e][b0 + lane];
            sq_row[s][lane] = qrow[e][b0 + lane];
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                atomicExch(&sh.sq_state[s], SQ_FULL);
            }
        };

        // this lane's column in chunk j of tile t is t * BN + (cw * CPW + j) * 32 + lane; the
        // norms are prefetched two tiles ahead so the load latency stays off the per-tile path
        const int cbase = cw * CPW * 32;
        const float* xp = D.xnorm + cbase + lane;
        int xrem = (int)n - (cbase + lane);     // > j * 32 while the lane's column of chunk j exists
        int crem = (int)n - cbase;              // columns left from the warp's first chunk
        float xa[CPW], xb[CPW];
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
            xa[j] = xrem > j * 32 ? xp[j * 32] : 0.f;
            xb[j] = xrem > BN + j * 32 ? xp[BN + j * 32] : 0.f;
        }
        bool aborted = false;
        for (int t = 0; t < ntiles; ++t) {
            const int b = t % NACC;
            float xc[CPW];
#pragma unroll
            for (int j = 0; j < CPW; ++j) xc[j] = xrem > 2 * BN + j * 32 ? xp[2 * BN + j * 32] : 0.f;
            // one lane waits, the whole warp follows its verdict (tcgen05.ld needs the full warp)
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&sh.acc_full[b], (t / NACC) & 1, err) ? 1 : 0;
            ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    atomicOr(err, ERR_TIMEOUT);
                    sh.abort = 1;
                }
                aborted = true;
                break;
            }
#pragma unroll
            for (int j = 0; j < CPW; ++j) bcol[e][j * 32 + lane] = fmaf(gamma, xa[j], gz);
            tc_fence_after();
#pragma unroll
            for (int j = 0; j < CPW; ++j) {
                uint32_t v[32];
                tmem_ld32_async(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + cbase + j * 32), v);
                tmem_wait_ld(v);
                if (j == CPW - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh.acc_empty[b]);   // the accumulator is in registers now
                } else {
                    __syncwarp();
                }
                const int cr = crem - j * 32;
                const uint32_t vmask = !live ? 0u : (cr >= 32 ? 0xFFFFFFFFu : (cr <= 0 ? 0u : ~(0xFFFFFFFFu >> cr)));
                // bit 31-k of a word is column k: two chains of 16 per word for instruction-level parallelism
                uint32_t s0 = 0u, s1 = 0u, b0 = 0u, b1 = 0u;
                const float4* bq = reinterpret_cast<const float4*>(&bcol[e][j * 32]);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const float4 B4 = bq[g], C4 = bq[g + 4];
                    const float Bk[4] = {B4.x, B4.y, B4.z, B4.w};
                    const float Ck[4] = {C4.x, C4.y, C4.z, C4.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const uint32_t va = v[g * 4 + h], vb = v[16 + g * 4 + h];
                        s0 = __funnelshift_l(va, s0, 1);
                        s1 = __funnelshift_l(vb, s1, 1);
                        b0 = __funnelshift_l(__float_as_uint(__fsub_rn(Bk[h], fabsf(__uint_as_float(va)))), b0, 1);
                        b1 = __funnelshift_l(__float_as_uint(__fsub_rn(Ck[h], fabsf(__uint_as_float(vb)))), b1, 1);
                    }
                }
                const uint32_t sa = __byte_perm(s1, s0, 0x5410);               // (s0 << 16) | s1
                const uint32_t ba = __byte_perm(b1, b0, 0x5410) & vmask;        // set: |t| > bound
                const uint32_t neg = __popc(sa & ba);
                lt += neg;
                gt += __popc(ba) - neg;
                uint32_t cm = vmask & ~ba;                                      // candidates
                unsigned bal = __ballot_sync(0xFFFFFFFFu, cm != 0u);
                if (bal) {
                    const uint32_t c0 = (uint32_t)(t * BN + cbase + j * 32);
                    do {
                        const int pos = qn + __popc(bal & ((1u << lane) - 1u));
                        if (cm) {
                            const int k = __clz(cm);
                            cm &= ~(0x80000000u >> k);
                            qpt[e][pos] = c0 + (uint32_t)k;
                            qrow[e][pos] = (uint8_t)row;
                        }
                        qn += __popc(bal);
                        if (qn >= 32) {
                            hand_off(qn - 32);
                            qn -= 32;
                        }
                        bal = __ballot_sync(0xFFFFFFFFu, cm != 0u);
                    } while (bal);
                }
            }
            __syncwarp();   // bcol is rewritten next tile
#pragma unroll
            for (int j = 0; j < CPW; ++j) {
                xa[j] = xb[j];
                xb[j] = xc[j];
            }
            xp += BN;
            xrem -= BN;
            crem -= BN;
        }
        if (!aborted && qn > 0) settle(&qpt[e][0], &qrow[e][0], qn);
        // the four warps of a lane quarter each counted a quarter of the columns
        partial_lt[e][lane] = lt;
        partial_gt[e][lane] = gt;
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            atomicAdd(&sh.epi_done, 1);   // every batch of this warp is in the ring by now
        }
    } else {
        // ---- settle warps: take full ring slots until the counting warps are done ----------
        // The wait is bounded by progress: it gives up only when the MMA issuer has not moved
        // for 2e9 cycles while batches may still come.
        long long t0 = clock64();
        int seen = -1;
        for (;;) {
            int s = -1, fin = 0;
            if (lane == 0) {
                for (int i = 0; i < NSLOT; ++i) {
                    if (*(volatile int*)&sh.sq_state[i] == SQ_FULL &&
                        atomicCAS(&sh.sq_state[i], SQ_FULL, SQ_SETTLING) == SQ_FULL) {
                        s = i;
                        break;
                    }
                }
                if (s >= 0) {
                    __threadfence_block();
                } else if (*(volatile int*)&sh.abort) {
                    fin = 1;
                } else if (*(volatile int*)&sh.epi_done == NEPI) {
                    __threadfence_block();
                    fin = 1;   // no slot is FILLING any more; a FULL one is taken next pass
                    for (int i = 0; i < NSLOT; ++i)
                        if (*(volatile int*)&sh.sq_state[i] == SQ_FULL) fin = 0;
                } else {
                    const int mt = *(volatile int*)&sh.mma_tiles;
                    const long long now = clock64();
                    if (mt != seen) {
                        seen = mt;
                        t0 = now;
                    } else if (now - t0 > 2000000000LL) {
                        atomicOr(err, ERR_TIMEOUT);
                        sh.abort = 1;
                        fin = 1;
                    }
                }
            }
            s = __shfl_sync(0xFFFFFFFFu, s, 0);
            fin = __shfl_sync(0xFFFFFFFFu, fin, 0);
            if (s >= 0) {
                settle(sq_pt[s], sq_row[s], 32);
                if (lane == 0) {
                    __threadfence_block();
                    atomicExch(&sh.sq_state[s], SQ_FREE);
                }
                continue;
            }
            if (fin) break;
            __nanosleep(256);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp >= 2 && warp < 6) {
        const int e = warp - 2;   // warps e, e + 4, e + 8, e + 12 read the same TMEM lanes
        const int row = (warp & 3) * 32 + lane;
        if (row < T.nj && !sh.abort) {
            const long long l2 = (long long)partial_lt[e][lane] + partial_lt[e + 4][lane] + partial_lt[e + 8][lane] +
                                 partial_lt[e + 12][lane] + cand_lt[row];
            const long long g2 = (long long)partial_gt[e][lane] + partial_gt[e + 4][lane] + partial_gt[e + 8][lane] +
                                 partial_gt[e + 12][lane] + cand_gt[row];
            const int64_t le = n - g2, ge = n - l2;
            const int64_t cmin = le < ge ? le : ge;
            res[rows[row].roff] = ResDev{(double)cmin / (double)n, cmin};
        }
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NACC * BN) : "memory");
    }
}

__global__ void k_build_planes(const float* __restrict__ X32, int64_t n, int d, int ldx, int kp,
                               uint16_t* __restrict__ Xbf)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * kp) return;
    const int64_t i = e / kp;
    const int k = (int)(e - i * kp);
    float hi = 0.f, lo = 0.f;
    if (k < d) {
        const float x = X32[i * ldx + k];
        hi = bf16_val(bf16_bits(x));
        lo = x - hi;
    } else if (k == d || k == d + 1) {
        hi = 1.0f;   // multiplies the folded -u'z parts of the direction planes
    }
    Xbf[i * 2 * kp + k] = bf16_bits(hi);
    Xbf[i * 2 * kp + kp + k] = bf16_bits(lo);
}

}  // namespace

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

namespace {

// ring stages: 2 x 64 KB (K extent 64, 256 points; 128, 128 points), 4 x 32 KB (64, 128 points)
int tc_stages(int kp, int bn) { return (kp == 64 && bn == 128) ? 4 : 2; }

size_t tc_smem_bytes(int kp, int bn)
{
    const size_t nchunk = (size_t)kp / 64;
    return 1024 /* alignment slack */ + 2 * nchunk * plane_bytes_rows(BM) +
           (size_t)tc_stages(kp, bn) * 2 * nchunk * plane_bytes_rows(bn);
}

// Failure-path check: one thread waits on an mbarrier that nothing will complete,
// with the same bounded wait as the tensor-core kernel but a caller-set limit.
__global__ void k_wait_probe(int* err, long long limit_cycles)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const long long t0 = clock64();
    bool ok = false;
    while (!(ok = mbar_test(&bar, 0))) {
        if (clock64() - t0 > limit_cycles) break;
    }
    if (!ok) atomicOr(err, ERR_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_probe(int* err, long long limit_cycles, cudaStream_t st)
{
    k_wait_probe<<<1, 32, 0, st>>>(err, limit_cycles);
    return cudaGetLastError();
}

float band_gamma_tc(int kp)
{
    // split residuals 3 * 2^-16 |u||x| (with 1% slack), FP32 accumulation of 3*kp products at most one
    // 2^-23 relative error each, the 2^-24 rounding of y_z's three BF16 parts; times 1.25
    const double g = 3.03 * 0x1p-16 + 3.03 * (double)kp * 0x1p-23 + 0x1p-22;
    return (float)(1.25 * g);
}

__host__ __device__ float band_coef_ff(int d)
{
    // compensated FP32 dot product of d terms: the rounding errors of the gathered error terms,
    // at most (2d^2 + 4d + 8) 2^-48 sum|u x|; y_z's FP64 evaluation and its FP32 pair, at most
    // (d + 8) 2^-52 |u'z|; |u| <= 1 + 2^-20 covered by the 1% slack
    const double dd = (double)d;
    return (float)(((2.0 * dd * dd + 4.0 * dd + 8.0) * 0x1p-48 + (dd + 8.0) * 0x1p-52) * 1.01);
}

bool hd_tc_supported(int d) { return d >= 1 && d + 2 <= 128; }

cudaError_t launch_build_bf16_planes(const float* X32, int64_t n, int d, int ldx, int kp, uint16_t* Xbf,
                                     cudaStream_t st)
{
    const int64_t total = n * kp;
    const int nt = 256;
    k_build_planes<<<(unsigned)((total + nt - 1) / nt), nt, 0, st>>>(X32, n, d, ldx, kp, Xbf);
    return cudaGetLastError();
}

int tc_tile_n(int kp, int want)
{
    // 256 points per tile for a K extent of 64 (a 128 x 256 x 16 MMA runs at the full tensor rate, 128 x 128 x 16
    // does not), unless 128 is asked for; 128 for a K extent of 128 (two 256-point stages would not fit)
    if (kp <= 64) return want == 128 ? 128 : 256;
    return 128;
}

cudaError_t encode_tc_map(const DsDev& ds_host, int bn, CUtensorMap* out)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int kp = ds_host.kp;
    if (kp != 64 && kp != 128) return cudaErrorInvalidValue;
    if (ds_host.n > 0x7FFFFFFF) return cudaErrorInvalidValue;   // point indices and TMA rows are 32-bit
    // the BF16 planes of this dataset only (no multicast): rows of 2 kp elements, boxes of 64 x BN
    const cuuint64_t gdim[2] = {(cuuint64_t)(2 * kp), (cuuint64_t)ds_host.n};
    const cuuint64_t gstride[1] = {(cuuint64_t)(2 * kp) * sizeof(uint16_t)};
    if (bn != tc_tile_n(kp, bn)) return cudaErrorInvalidValue;
    const cuuint32_t box[2] = {64, (cuuint32_t)bn};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)ds_host.Xbf, gdim, gstride, box, estride,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_hd_tc(const TaskDev* tasks, int ntasks, int kp, int bn, const SlotDev* slots,
                         const DsDev* ds_dev, const CUtensorMap* maps, const float* U, const double* yz,
                         const double* z64, ResDev* res, int64_t* band_out, int* err, cudaStream_t st)
{
    if (ntasks <= 0) return cudaSuccess;
    if (kp != 64 && kp != 128) return cudaErrorInvalidValue;
    if (bn != tc_tile_n(kp, bn)) return cudaErrorInvalidValue;
    const size_t smem = tc_smem_bytes(kp, bn);
    auto kern = bn == 256 ? k_hd_tc<256> : k_hd_tc<128>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    kern<<<ntasks, NTHREADS, smem, st>>>(maps, tasks, slots, ds_dev, U, yz, z64, res, band_out, err,
                                         band_gamma_tc(kp), tc_stages(kp, bn));
    return cudaGetLastError();
}

}  // namespace rrs
