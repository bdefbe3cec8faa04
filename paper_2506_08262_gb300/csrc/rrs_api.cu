// Host runtime behind the C ABI of include/rrs.h: dataset registry, device
// memory accounting, per-call workspace and the refinement-round pipeline
// (Alg. 4: generate -> project + univariate depth -> minimum and pole update,
// r times; queries and requests are independent work items of every launch).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/rrs.h"
#include "rrs_internal.h"
#include "rrs_ctx.h"

using namespace rrs;

namespace {

thread_local std::string g_last_error;

rrs_status fail(rrs_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

// On failure the runtime's pending error is cleared so that it cannot surface
// in an unrelated later call.
#define CUDA_TRY(expr)                                                                     \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return fail(RRS_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), \
                        __FILE__, __LINE__);                                               \
        }                                                                                  \
    } while (0)

// Opt-in host trace (RRS_TRACE=1) for locating failures in the runtime.
void trace(const char* fmt, ...)
{
    static const bool on = getenv("RRS_TRACE") && getenv("RRS_TRACE")[0] == '1';
    if (!on) return;
    va_list ap;
    va_start(ap, fmt);
    fprintf(stderr, "[rrs] ");
    vfprintf(stderr, fmt, ap);
    fprintf(stderr, "\n");
    fflush(stderr);
    va_end(ap);
}

int padded_ldx(int d)
{
    int l = (d + 3) & ~3;
    if (((l / 4) & 1) == 0) l += 4;  // odd number of float4 per row: conflict-free staging
    return l;
}

int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }



// A bump allocator over one device allocation.
struct Carve {
    char* base = nullptr;
    size_t off = 0;
    size_t cap = 0;
    template <typename T>
    T* take(size_t count)
    {
        off = (size_t)align_up((int64_t)off, 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += sizeof(T) * (count ? count : 1);
        return p;
    }
};

}  // namespace

void rrs::set_last_error(const char* msg) { g_last_error = msg; }


namespace {

cudaEvent_t pooled_event(rrs_ctx* c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one launch with events when profiling is on (not during graph capture).
struct StageTimer {
    rrs_ctx* c;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageTimer(rrs_ctx* c_, int stage_, cudaStream_t st_, bool capturing) : c(c_), stage(stage_), st(st_)
    {
        if (c->profiling && !capturing) {
            a = pooled_event(c);
            cudaEventRecord(a, st);
        }
    }
    ~StageTimer()
    {
        if (a) {
            cudaEvent_t b = pooled_event(c);
            cudaEventRecord(b, st);
            c->marks.push_back(rrs_ctx::Mark{stage, a, b});
        }
    }
};

bool budget_ok(rrs_ctx* c, uint64_t extra) { return c->budget == 0 || c->used + extra <= c->budget; }

struct Plan {
    // host copies of everything the kernels read
    std::vector<DsDev> ds;
    std::vector<SlotDev> slots;
    std::vector<TaskDev> gen_tasks, hd_tasks;
    std::vector<std::vector<TaskDev>> pd_tasks;       // one list per (shared-memory class, group, d class)
    std::vector<size_t> pd_smem;                      // dynamic shared memory of each list: its largest need
    std::vector<int> pd_group, pd_variant;
    std::vector<int> pd_keys_ds;                      // d > 16: dataset whose keys k_keys forms first (-1: none)
    std::vector<int> pd_keys_chunk;                   // tasks per keys launch (bounded by the keys scratch)
    std::vector<int32_t> argmin_list;
    // active prefix lengths per round
    std::vector<int> n_gen, n_hd, n_arg;
    std::vector<std::vector<int>> n_pd;
    int rmax = 0;
    int max_ldx = 4;
    int64_t tot_ldx = 0, tot_d = 0, tot_u = 0, tot_m = 0;
    // tensor-core halfspace tasks, one group per K extent of the planes (64 or 128), each group one launch
    // per round whatever the datasets: every task's CTA takes its dataset's tensor map from maps
    struct TcGroup {
        int kp = 0, bn = 0;   // K extent of the planes, points per tile
        std::vector<TaskDev> tasks;
        std::vector<int> n;   // active prefix per round
        TaskDev* d = nullptr;
    };
    std::vector<TcGroup> tc;
    std::vector<CUtensorMap> maps;     // one per dataset row (encoded for datasets with tensor-core tasks)
    CUtensorMap* d_maps = nullptr;
    // selection-kernel group size: autotuned choices and an explicit override (tuning probes)
    const std::map<std::tuple<int64_t, int, int>, int>* tune = nullptr;
    const std::map<std::pair<int64_t, int>, int>* tc_tune = nullptr;   // (n, kp) -> points per tile
    int force_group = 0;
    // device pointers (after carving)
    DsDev* d_ds = nullptr;
    SlotDev* d_slots = nullptr;
    TaskDev *d_gen = nullptr, *d_hd = nullptr;
    std::vector<TaskDev*> d_pd;
    int32_t* d_arg = nullptr;
    float *z32 = nullptr, *poles = nullptr, *U = nullptr, *keys = nullptr;
    size_t keys_floats = 0;
    double *z64 = nullptr, *yz = nullptr;
    ResDev* res = nullptr;
};

struct ReqView {
    const Dataset* dset;
    int ds_index;
    const void* Z;
    int64_t nq;
    int32_t dtype;
    int32_t kind;
    int32_t k, r;
    float alpha;
    uint64_t seed;
    double* depth_out;
    int64_t* count_out;
    int32_t* best_out;
    int32_t* choice_out;
    int64_t q_base;
    int32_t precision;   // RRS_PREC_* for halfspace requests
};

rrs_status validate_params(int32_t kind, int32_t k, int32_t r, double alpha, int32_t dtype, int32_t precision)
{
    if (kind < 0 || kind > 2) return fail(RRS_ERR_INVALID_ARG, "unknown depth kind %d", kind);
    if (r < 1 || k < r) return fail(RRS_ERR_INVALID_ARG, "need n_dirs >= n_refinements >= 1 (k=%d r=%d)", k, r);
    if (!(alpha > 0.0) || alpha > 1.0) return fail(RRS_ERR_INVALID_ARG, "cap_shrink must be in (0, 1]");
    if (dtype != RRS_F32 && dtype != RRS_F64) return fail(RRS_ERR_INVALID_ARG, "unknown dtype %d", dtype);
    if (precision != RRS_PREC_FP32_SIMT && precision != RRS_PREC_SPLIT_BF16X3)
        return fail(RRS_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (precision == RRS_PREC_SPLIT_BF16X3 && kind != RRS_HALFSPACE)
        return fail(RRS_ERR_INVALID_ARG, "split-BF16x3 precision serves halfspace depth only");
    return RRS_OK;
}

// Build the launch plan for a set of requests (requests sorted by r, descending).
rrs_status build_plan(const std::vector<ReqView>& reqs, Plan& P)
{
    std::vector<int> order(reqs.size());
    for (size_t i = 0; i < reqs.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return reqs[a].r > reqs[b].r; });
    std::map<const Dataset*, int> dsidx;
    for (int ri : order) {
        const ReqView& R = reqs[ri];
        if (!dsidx.count(R.dset)) {
            const Dataset& D = *R.dset;
            DsDev dd{};
            dd.X32 = D.X32;
            dd.Xt = D.Xt;
            dd.X64 = D.X64;
            dd.xnorm = D.xnorm;
            dd.Xbf = D.Xbf;
            dd.n = D.n;
            dd.d = D.d;
            dd.ldx = D.ldx;
            dd.kp = D.kp;
            dd.center = D.center;
            dd.cov = D.cov;
            dd.rc = D.rc;
            dsidx[R.dset] = (int)P.ds.size();
            P.ds.push_back(dd);
        }
    }
    // shared-memory classes group the selection launches; each launch requests the largest need of its
    // class, not the class bound, so small needs keep more of the SM's memory as L1
    const size_t classes[] = {24 * 1024, 48 * 1024, 72 * 1024, 110 * 1024, pdap_smem_limit()};
    std::map<std::tuple<size_t, int, int, int>, int> pd_index;
    auto pd_list = [&](size_t cls_bytes, size_t need, int group, int variant, int keys_ds) {
        auto key = std::make_tuple(cls_bytes, group, variant, keys_ds);
        auto it = pd_index.find(key);
        if (it != pd_index.end()) {
            P.pd_smem[it->second] = std::max(P.pd_smem[it->second], need);
            return it->second;
        }
        const int idx = (int)P.pd_tasks.size();
        pd_index[key] = idx;
        P.pd_tasks.emplace_back();
        P.pd_smem.push_back(need);
        P.pd_group.push_back(group);
        P.pd_variant.push_back(variant);
        P.pd_keys_ds.push_back(keys_ds);
        P.pd_keys_chunk.push_back(0);
        return idx;
    };
    struct SlotRounds {
        int r;
    };
    std::vector<int> slot_r;
    for (int ri : order) {
        const ReqView& R = reqs[ri];
        const Dataset& D = *R.dset;
        const int m = (R.k + R.r - 1) / R.r;
        int G = 0;
        int cls = -1;
        const bool tc = R.kind == RRS_HALFSPACE && R.precision == RRS_PREC_SPLIT_BF16X3;
        if (R.kind == RRS_HALFSPACE && !tc && D.ldx > 440)
            return fail(RRS_ERR_UNSUPPORTED, "FP32 halfspace kernel stages 128 rows of d floats; d=%d too large", D.d);
        if (R.kind != RRS_HALFSPACE) {
            if (D.n > PDAP_MAX_N) return fail(RRS_ERR_UNSUPPORTED, "n too large for the selection kernel");
            int want = P.force_group;
            if (!want && P.tune) {
                auto it = P.tune->find(std::make_tuple(D.n, D.ldx, m));
                if (it != P.tune->end()) want = it->second;
            }
            // resident keys when they fit shared memory, else keys formed once and read at every pass
            const PdapShape sh = pdap_shape((int)D.n, D.ldx, m, D.d, want);
            G = sh.group;
            // keys formed first by a keys kernel (d > 16, or keys outside shared memory): one list per
            // dataset, since a keys launch reads one X
            const int keys_ds = sh.keys_gemm ? dsidx[R.dset] : -1;
            for (size_t c : classes)
                if (sh.smem <= c) {
                    cls = pd_list(c, sh.smem, G, sh.variant, keys_ds);
                    break;
                }
            if (cls < 0) return fail(RRS_ERR_INTERNAL, "no shared-memory class for n=%lld", (long long)D.n);
        }
        const int s_first = (int)P.slots.size();
        for (int64_t q = 0; q < R.nq; ++q) {
            SlotDev S{};
            S.ds = dsidx[R.dset];
            S.kind = R.kind;
            S.m = m;
            S.r = R.r;
            S.alpha = R.alpha;
            S.d = D.d;
            S.ldx = D.ldx;
            S.zdtype = R.dtype;
            S.seed = R.seed;
            S.qctr = R.q_base + q;
            S.uoff = P.tot_u;
            S.roff = P.tot_m;
            S.zoff32 = P.tot_ldx;
            S.zoff64 = P.tot_d;
            S.zsrc = (const char*)R.Z + (size_t)q * D.d * (R.dtype == RRS_F32 ? 4 : 8);
            S.depth_out = R.depth_out ? R.depth_out + q : nullptr;
            S.count_out = R.count_out ? R.count_out + q : nullptr;
            S.best_out = R.best_out ? R.best_out + q : nullptr;
            S.choice_out = R.choice_out ? R.choice_out + q * R.r : nullptr;
            const int s = (int)P.slots.size();
            P.slots.push_back(S);
            slot_r.push_back(R.r);
            P.tot_u += (int64_t)m * D.ldx;
            P.tot_m += m;
            P.tot_ldx += D.ldx;
            P.tot_d += D.d;
            P.max_ldx = std::max(P.max_ldx, D.ldx);
            for (int j0 = 0; j0 < m; j0 += 128) P.gen_tasks.push_back(TaskDev{s, j0, std::min(128, m - j0), 0});
            if (R.kind == RRS_HALFSPACE) {
                if (!tc) {
                    const int cap = 64;   // directions per CTA of the FP32 kernel
                    const int nt = (m + cap - 1) / cap;
                    const int per = (m + nt - 1) / nt;
                    for (int j0 = 0; j0 < m; j0 += per) P.hd_tasks.push_back(TaskDev{s, j0, std::min(per, m - j0), 0});
                }
            } else {
                for (int j0 = 0; j0 < m; j0 += G) P.pd_tasks[cls].push_back(TaskDev{s, j0, std::min(G, m - j0), S.ds});
            }
            P.argmin_list.push_back(s);
        }
        if (tc) {
            // tensor-core tasks: 128 consecutive (query, direction) rows of this request, so the
            // accumulator's M dimension is filled across queries (task = first query slot, offset
            // into that query's directions, row count); one task list per K extent, and the dataset's
            // tensor map in the plan's map table
            const int dsi = dsidx[R.dset];
            const int kp = P.ds[dsi].kp;
            int want = 0;
            if (P.tc_tune) {
                auto it = P.tc_tune->find(std::make_pair(P.ds[dsi].n, kp));
                if (it != P.tc_tune->end()) want = it->second;
            }
            const int bn = tc_tile_n(kp, want);
            if (P.maps.size() < P.ds.size()) P.maps.resize(P.ds.size());
            if (P.ds[dsi].Xbf) {
                static const CUtensorMap zero{};
                if (!memcmp(&P.maps[dsi], &zero, sizeof zero) &&
                    encode_tc_map(P.ds[dsi], bn, &P.maps[dsi]) != cudaSuccess)
                    return fail(RRS_ERR_CUDA, "tensor map of dataset row %d", dsi);
            }
            size_t gi = 0;
            while (gi < P.tc.size() && (P.tc[gi].kp != kp || P.tc[gi].bn != bn)) ++gi;
            if (gi == P.tc.size()) {
                P.tc.emplace_back();
                P.tc.back().kp = kp;
                P.tc.back().bn = bn;
            }
            const int64_t rows = R.nq * (int64_t)m;
            for (int64_t g = 0; g < rows; g += 128)
                P.tc[gi].tasks.push_back(
                    TaskDev{s_first + (int)(g / m), (int)(g % m), (int)std::min<int64_t>(128, rows - g), 0});
        }
        P.rmax = std::max(P.rmax, R.r);
    }
    // active prefixes: slots are sorted by r descending, so round l uses the slots with r > l
    auto prefix = [&](const std::vector<TaskDev>& t, std::vector<int>& out) {
        out.assign(P.rmax, 0);
        for (int l = 0; l < P.rmax; ++l) {
            int c = 0;
            while (c < (int)t.size() && slot_r[t[c].slot] > l) ++c;
            out[l] = c;
        }
    };
    prefix(P.gen_tasks, P.n_gen);
    prefix(P.hd_tasks, P.n_hd);
    for (auto& g : P.tc) prefix(g.tasks, g.n);
    P.n_pd.resize(P.pd_tasks.size());
    for (size_t c = 0; c < P.pd_tasks.size(); ++c) prefix(P.pd_tasks[c], P.n_pd[c]);
    // keys scratch: one chunk of the largest keys list at a time, at most KEYS_SCRATCH_BYTES
    constexpr size_t KEYS_SCRATCH_BYTES = 256u << 20;
    for (size_t c = 0; c < P.pd_tasks.size(); ++c) {
        if (P.pd_keys_ds[c] < 0 || P.pd_tasks[c].empty()) continue;
        const int n = (int)P.ds[P.pd_keys_ds[c]].n;
        const size_t per = pdap_keys_bytes(n, P.pd_group[c], 1);
        const int chunk = (int)std::max<size_t>(1, std::min<size_t>(P.pd_tasks[c].size(), KEYS_SCRATCH_BYTES / per));
        P.pd_keys_chunk[c] = chunk;
        P.keys_floats = std::max(P.keys_floats, pdap_keys_bytes(n, P.pd_group[c], chunk) / sizeof(float));
    }
    P.n_arg.assign(P.rmax, 0);
    for (int l = 0; l < P.rmax; ++l) {
        int c = 0;
        while (c < (int)P.argmin_list.size() && slot_r[P.argmin_list[c]] > l) ++c;
        P.n_arg[l] = c;
    }
    return RRS_OK;
}

size_t carve_plan(Plan& P, Carve& C)
{
    P.d_ds = C.take<DsDev>(P.ds.size());
    P.d_slots = C.take<SlotDev>(P.slots.size());
    P.d_gen = C.take<TaskDev>(P.gen_tasks.size());
    P.d_hd = C.take<TaskDev>(P.hd_tasks.size());
    for (auto& g : P.tc) g.d = C.take<TaskDev>(g.tasks.size());
    P.d_maps = P.maps.empty() ? nullptr : C.take<CUtensorMap>(P.maps.size());
    P.d_pd.resize(P.pd_tasks.size());
    for (size_t c = 0; c < P.pd_tasks.size(); ++c) P.d_pd[c] = C.take<TaskDev>(P.pd_tasks[c].size());
    P.d_arg = C.take<int32_t>(P.argmin_list.size());
    P.z32 = C.take<float>(P.tot_ldx);
    P.poles = C.take<float>(2 * P.tot_ldx);
    P.z64 = C.take<double>(P.tot_d);
    P.U = C.take<float>(P.tot_u);
    P.yz = C.take<double>(P.tot_m);
    P.res = C.take<ResDev>(P.tot_m);
    P.keys = P.keys_floats ? C.take<float>(P.keys_floats) : nullptr;
    return C.off;
}

// Upload the plan's host tables (slots, tasks) into the carved workspace.
rrs_status upload_plan(rrs_ctx* ctx, Plan& P, cudaStream_t st)
{
    (void)ctx;
    auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        if (!bytes) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    CUDA_TRY(up(P.d_ds, P.ds.data(), P.ds.size() * sizeof(DsDev)));
    CUDA_TRY(up(P.d_slots, P.slots.data(), P.slots.size() * sizeof(SlotDev)));
    CUDA_TRY(up(P.d_gen, P.gen_tasks.data(), P.gen_tasks.size() * sizeof(TaskDev)));
    CUDA_TRY(up(P.d_hd, P.hd_tasks.data(), P.hd_tasks.size() * sizeof(TaskDev)));
    for (auto& g : P.tc) CUDA_TRY(up(g.d, g.tasks.data(), g.tasks.size() * sizeof(TaskDev)));
    if (P.d_maps) CUDA_TRY(up(P.d_maps, P.maps.data(), P.maps.size() * sizeof(CUtensorMap)));
    for (size_t c = 0; c < P.pd_tasks.size(); ++c)
        CUDA_TRY(up(P.d_pd[c], P.pd_tasks[c].data(), P.pd_tasks[c].size() * sizeof(TaskDev)));
    CUDA_TRY(up(P.d_arg, P.argmin_list.data(), P.argmin_list.size() * sizeof(int32_t)));
    return RRS_OK;
}

// Enqueue the whole refinement pipeline of a plan.
rrs_status enqueue_rounds(rrs_ctx* ctx, Plan& P, cudaStream_t st, bool capturing = false)
{
    const int64_t T = P.tot_ldx;
    {
        StageTimer t(ctx, RRS_STAGE_PREP, st, capturing);
        CUDA_TRY(launch_prep(P.d_slots, (int)P.slots.size(), P.d_ds, P.z32, P.z64, P.poles, st));
        ctx->launches++;
        ctx->stage_launches[RRS_STAGE_PREP]++;
    }
    for (int l = 0; l < P.rmax; ++l) {
        float* cur = P.poles + (l & 1) * T;
        float* nxt = P.poles + ((l + 1) & 1) * T;
        if (P.n_gen[l] > 0) {
            StageTimer t(ctx, RRS_STAGE_GEN, st, capturing);
            CUDA_TRY(launch_gen(P.d_gen, P.n_gen[l], P.d_slots, cur, P.z64, P.U, P.yz, l, P.max_ldx, st));
            ctx->launches++;
            ctx->stage_launches[RRS_STAGE_GEN]++;
        }
        if (P.n_hd[l] > 0) {
            StageTimer t(ctx, RRS_STAGE_HD_SIMT, st, capturing);
            CUDA_TRY(launch_hd_simt(P.d_hd, P.n_hd[l], P.max_ldx, P.d_slots, P.d_ds, P.U, P.yz, P.z64, P.res,
                                    nullptr, ctx->d_err, st));
            ctx->stage_launches[RRS_STAGE_HD_SIMT]++;
            ctx->launches++;
        }
        for (auto& g : P.tc) {
            if (g.n[l] <= 0) continue;
            StageTimer t(ctx, RRS_STAGE_HD_TC, st, capturing);
            CUDA_TRY(launch_hd_tc(g.d, g.n[l], g.kp, g.bn, P.d_slots, P.d_ds, P.d_maps, P.U, P.yz, P.z64, P.res,
                                  nullptr, ctx->d_err, st));
            ctx->stage_launches[RRS_STAGE_HD_TC]++;
            ctx->launches++;
        }
        for (size_t c = 0; c < P.pd_tasks.size(); ++c) {
            if (P.n_pd[c][l] <= 0) continue;
            if (P.pd_keys_ds[c] < 0) {
                StageTimer t(ctx, RRS_STAGE_PDAP, st, capturing);
                CUDA_TRY(launch_pdap(P.d_pd[c], P.n_pd[c][l], P.pd_smem[c], P.pd_group[c], P.pd_variant[c], P.d_slots,
                                     P.d_ds, P.U, P.yz, P.res, ctx->d_err, st));
                ctx->launches += PDAP_LAUNCH_KERNELS;
                ctx->stage_launches[RRS_STAGE_PDAP]++;
                continue;
            }
            // keys by the tiled GEMM, then the selection on them, one scratch-sized chunk at a time
            const int total = P.n_pd[c][l], chunk = P.pd_keys_chunk[c];
            for (int t0 = 0; t0 < total; t0 += chunk) {
                const int cnt = std::min(chunk, total - t0);
                {
                    StageTimer t(ctx, RRS_STAGE_KEYS, st, capturing);
                    CUDA_TRY(launch_pdap_keys(P.d_pd[c] + t0, cnt, P.pd_group[c], P.d_slots, P.d_ds,
                                              P.ds[P.pd_keys_ds[c]], P.U, P.keys, st));
                }
                StageTimer t(ctx, RRS_STAGE_PDAP, st, capturing);
                CUDA_TRY(launch_pdap(P.d_pd[c] + t0, cnt, P.pd_smem[c], P.pd_group[c], P.pd_variant[c], P.d_slots,
                                     P.d_ds, P.U, P.yz, P.res, ctx->d_err, st, P.keys));
                ctx->launches += 1 + PDAP_LAUNCH_KERNELS;
                ctx->stage_launches[RRS_STAGE_KEYS]++;
                ctx->stage_launches[RRS_STAGE_PDAP]++;
            }
        }
        if (P.n_arg[l] > 0) {
            StageTimer t(ctx, RRS_STAGE_ARGMIN, st, capturing);
            CUDA_TRY(launch_argmin(P.d_slots, P.d_arg, P.n_arg[l], P.U, P.res, cur, nxt, l, 0, st));
            ctx->launches++;
            ctx->stage_launches[RRS_STAGE_ARGMIN]++;
        }
    }
    return RRS_OK;
}

rrs_status check_device_errors(rrs_ctx* ctx, cudaStream_t st)
{
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        if (h & ERR_TIMEOUT) return fail(RRS_ERR_TIMEOUT, "a bounded device-side wait gave up (flags 0x%x)", h);
        return fail(RRS_ERR_INTERNAL, "device-side error flags 0x%x", h);
    }
    return RRS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char* rrs_status_string(rrs_status s)
{
    switch (s) {
    case RRS_OK: return "ok";
    case RRS_ERR_INVALID_ARG: return "invalid argument";
    case RRS_ERR_NOT_FOUND: return "dataset not found";
    case RRS_ERR_BUDGET: return "device memory budget exceeded";
    case RRS_ERR_CUDA: return "CUDA error";
    case RRS_ERR_TIMEOUT: return "device-side wait timed out";
    case RRS_ERR_INTERNAL: return "internal error";
    case RRS_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
    }
}

const char* rrs_last_error(void) { return g_last_error.c_str(); }

rrs_status rrs_create(rrs_ctx** out, int32_t device, uint64_t hbm_budget_bytes)
{
    if (!out) return fail(RRS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(RRS_ERR_INVALID_ARG, "device %d out of range (%d)", device, ndev);
    CUDA_TRY(cudaSetDevice(device));
    std::unique_ptr<rrs_ctx> c(new rrs_ctx);
    c->device = device;
    c->budget = hbm_budget_bytes;
    CUDA_TRY(cudaMalloc(&c->d_err, sizeof(int)));
    CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
    *out = c.release();
    return RRS_OK;
}

rrs_status rrs_destroy(rrs_ctx* ctx)
{
    if (!ctx) return RRS_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->datasets) {
        cudaFree(kv.second.X32);
        cudaFree(kv.second.Xt);
        cudaFree(kv.second.X64);
        cudaFree(kv.second.xnorm);
        cudaFree(kv.second.Xbf);
        cudaFree(kv.second.center);
    }
    for (auto& g : ctx->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        cudaFree(g.ws);
    }
    for (auto& m : ctx->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    cudaFree(ctx->d_err);
    delete ctx;
    return RRS_OK;
}

rrs_status rrs_register_dataset(rrs_ctx* ctx, const void* X, int64_t n, int32_t d, int32_t dtype, int32_t x_on_device,
                                int64_t* dataset_id_out)
{
    if (!ctx || !X || !dataset_id_out) return fail(RRS_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || d < 1 || d > 1024) return fail(RRS_ERR_INVALID_ARG, "need n >= 1 and 1 <= d <= 1024");
    if (dtype != RRS_F32 && dtype != RRS_F64) return fail(RRS_ERR_INVALID_ARG, "unknown dtype");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    Dataset D;
    D.n = n;
    D.d = d;
    D.ldx = padded_ldx(d);
    const size_t esz = dtype == RRS_F32 ? 4 : 8;
    const size_t b32 = sizeof(float) * (size_t)n * D.ldx, b64 = dtype == RRS_F64 ? sizeof(double) * n * d : 0,
                 bn = sizeof(float) * n;
    const bool want_cov = d <= RRS_COV_MAX_D;
    const size_t bmom = sizeof(float) * ((size_t)d + (want_cov ? (size_t)d * d : 0) + 1);
    // the rows again in 32-row tiles for the selection kernels' projection pass (d <= 16: the kernels that
    // hold directions in registers), which streams X once per CTA and is bound by the cache lines its loads touch
    const size_t bt = d <= 16 ? sizeof(float) * tile_rows_floats(n, D.ldx) : 0;
    D.bytes = b32 + bt + b64 + bn + bmom;
    if (!budget_ok(ctx, D.bytes)) return fail(RRS_ERR_BUDGET, "dataset needs %zu bytes", D.bytes);
    void* staged = nullptr;
    const void* src = X;
    cudaStream_t st = 0;
    if (!x_on_device) {
        CUDA_TRY(cudaMalloc(&staged, esz * n * d));
        CUDA_TRY(cudaMemcpy(staged, X, esz * n * d, cudaMemcpyHostToDevice));
        src = staged;
    }
    cudaError_t e = cudaMalloc(&D.X32, b32);
    if (e == cudaSuccess && bt) e = cudaMalloc(&D.Xt, bt);
    if (e == cudaSuccess && b64) e = cudaMalloc(&D.X64, b64);
    if (e == cudaSuccess) e = cudaMalloc(&D.xnorm, bn);
    if (e == cudaSuccess) e = cudaMalloc(&D.center, bmom);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = launch_convert_dataset(src, dtype, n, d, D.ldx, D.X32, D.X64, D.xnorm, ctx->d_err, st);
    if (e == cudaSuccess && D.Xt) {
        e = launch_tile_rows(D.X32, n, D.ldx, D.Xt, st);
        ctx->launches++;
    }
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&bad, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    ctx->launches++;
    if (e == cudaSuccess && !bad) {
        D.cov = want_cov ? D.center + d : nullptr;
        float* rc_dev = D.center + d + (want_cov ? (size_t)d * d : 0);
        e = launch_moments(D.X32, n, d, D.ldx, D.center, D.cov, rc_dev, st);
        if (e == cudaSuccess) e = cudaMemcpy(&D.rc, rc_dev, sizeof(float), cudaMemcpyDeviceToHost);
        ctx->launches += 3;
    }
    cudaFree(staged);
    if (e != cudaSuccess || bad) {
        cudaGetLastError();
        cudaFree(D.X32);
        cudaFree(D.Xt);
        cudaFree(D.X64);
        cudaFree(D.xnorm);
        cudaFree(D.center);
        if (e != cudaSuccess) return fail(RRS_ERR_CUDA, "dataset upload failed: %s", cudaGetErrorString(e));
        return fail(RRS_ERR_INVALID_ARG, "X holds a non-finite value or one of magnitude >= 2^64");
    }
    ctx->used += D.bytes;
    const int64_t id = ctx->next_id++;
    ctx->datasets[id] = D;
    *dataset_id_out = id;
    return RRS_OK;
}

rrs_status rrs_free(rrs_ctx* ctx, int64_t dataset_id)
{
    if (!ctx) return fail(RRS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->datasets.find(dataset_id);
    if (it == ctx->datasets.end()) return fail(RRS_ERR_NOT_FOUND, "no dataset %lld", (long long)dataset_id);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    cudaFree(it->second.X32);
    cudaFree(it->second.Xt);
    cudaFree(it->second.X64);
    cudaFree(it->second.xnorm);
    cudaFree(it->second.Xbf);
    cudaFree(it->second.center);
    ctx->used -= it->second.bytes;
    ctx->datasets.erase(it);
    return RRS_OK;
}

}  // extern "C"

// Lazily build the BF16 planes of a dataset for the tensor-core path.
rrs_status rrs::ensure_bf16_planes(rrs_ctx* ctx, Dataset& D)
{
    if (D.Xbf) return RRS_OK;
    if (!hd_tc_supported(D.d)) return fail(RRS_ERR_UNSUPPORTED, "tensor-core path does not support d=%d", D.d);
    const int kp = (int)align_up(D.d + 2, 64);
    const size_t bytes = sizeof(uint16_t) * 2 * (size_t)kp * D.n;
    if (!budget_ok(ctx, bytes)) return fail(RRS_ERR_BUDGET, "BF16 planes need %zu bytes", bytes);
    CUDA_TRY(cudaMalloc(&D.Xbf, bytes));
    CUDA_TRY(launch_build_bf16_planes(D.X32, D.n, D.d, D.ldx, kp, D.Xbf, 0));
    CUDA_TRY(cudaDeviceSynchronize());
    ctx->launches++;
    D.kp = kp;
    D.bytes += bytes;
    ctx->used += bytes;
    return RRS_OK;
}

// Cached graphs replay the kernel choices of their capture: a changed choice drops them (after the device is
// idle, so none is in flight).
static void drop_graphs(rrs_ctx* ctx)
{
    if (ctx->graphs.empty()) return;
    cudaDeviceSynchronize();
    for (auto& g : ctx->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        cudaFree(g.ws);
    }
    ctx->graphs.clear();
    cudaGetLastError();
}

static rrs_status run_requests(rrs_ctx* ctx, std::vector<ReqView>& reqs, cudaStream_t st, int force_group = 0)
{
    Plan P;
    P.tune = &ctx->pd_tune;
    P.tc_tune = &ctx->tc_tune;
    P.force_group = force_group;
    rrs_status s = build_plan(reqs, P);
    if (s != RRS_OK) return s;
    if (P.slots.empty()) return RRS_OK;
    Carve sizing;
    const size_t bytes = carve_plan(P, sizing);
    if (!budget_ok(ctx, bytes)) return fail(RRS_ERR_BUDGET, "call workspace needs %zu bytes", bytes);
    void* ws = nullptr;
    CUDA_TRY(cudaMallocAsync(&ws, bytes, st));
    Carve C;
    C.base = (char*)ws;
    C.cap = bytes;
    carve_plan(P, C);
    s = upload_plan(ctx, P, st);
    if (s == RRS_OK) s = enqueue_rounds(ctx, P, st);
    cudaFreeAsync(ws, st);
    return s;
}

extern "C" {

rrs_status rrs_depth(rrs_ctx* ctx, int64_t dataset_id, const void* Z, int64_t n_queries, int32_t dtype,
                     int32_t z_on_device, int32_t kind, int32_t n_dirs, int32_t n_refinements, double cap_shrink,
                     uint64_t seed, int32_t precision, double* depth_out, int64_t* count_out, int32_t* best_out,
                     int32_t* round_choice_out, int32_t out_on_device, void* stream)
{
    if (!ctx) return fail(RRS_ERR_INVALID_ARG, "NULL context");
    rrs_status s = validate_params(kind, n_dirs, n_refinements, cap_shrink, dtype, precision);
    if (s != RRS_OK) return s;
    if (n_queries < 0) return fail(RRS_ERR_INVALID_ARG, "n_queries < 0");
    if (n_queries > 0 && (!Z || !depth_out)) return fail(RRS_ERR_INVALID_ARG, "Z and depth_out are required");
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->datasets.find(dataset_id);
    if (it == ctx->datasets.end()) return fail(RRS_ERR_NOT_FOUND, "no dataset %lld", (long long)dataset_id);
    if (n_queries == 0) return RRS_OK;
    CUDA_TRY(cudaSetDevice(ctx->device));
    Dataset& D = it->second;
    if (precision == RRS_PREC_SPLIT_BF16X3) {
        s = ensure_bf16_planes(ctx, D);
        if (s != RRS_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t esz = dtype == RRS_F32 ? 4 : 8;
    const size_t zbytes = esz * (size_t)n_queries * D.d;
    // device staging for host inputs / outputs
    void* zdev = nullptr;
    char* outdev = nullptr;
    const size_t r = (size_t)n_refinements;
    const size_t ob_depth = 8 * n_queries, ob_count = 8 * n_queries, ob_best = 4 * n_queries,
                 ob_choice = 4 * n_queries * r;
    const size_t obytes = ob_depth + ob_count + ob_best + ob_choice + 64;
    if (!z_on_device) {
        CUDA_TRY(cudaMallocAsync(&zdev, zbytes, st));
        CUDA_TRY(cudaMemcpyAsync(zdev, Z, zbytes, cudaMemcpyHostToDevice, st));
    }
    const void* zsrc = z_on_device ? Z : zdev;
    CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
    CUDA_TRY(launch_check_finite(zsrc, dtype, (int64_t)n_queries * D.d, ctx->d_err, st));
    ctx->launches++;
    ReqView R{};
    R.dset = &D;
    R.Z = zsrc;
    R.nq = n_queries;
    R.dtype = dtype;
    R.kind = kind;
    R.k = n_dirs;
    R.r = n_refinements;
    R.alpha = (float)cap_shrink;
    R.seed = seed;
    R.q_base = 0;
    R.precision = precision;
    if (out_on_device) {
        R.depth_out = depth_out;
        R.count_out = count_out;
        R.best_out = best_out;
        R.choice_out = round_choice_out;
    } else {
        CUDA_TRY(cudaMallocAsync((void**)&outdev, obytes, st));
        R.depth_out = (double*)outdev;
        R.count_out = (int64_t*)(outdev + ob_depth);
        R.best_out = (int32_t*)(outdev + ob_depth + ob_count);
        R.choice_out = (int32_t*)(outdev + ob_depth + ob_count + ob_best);
    }
    // the finiteness check must pass before any compute is trusted: read it now
    int bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (bad) {
        cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st);
        if (zdev) cudaFreeAsync(zdev, st);
        if (outdev) cudaFreeAsync(outdev, st);
        cudaStreamSynchronize(st);
        return fail(RRS_ERR_INVALID_ARG, "Z holds a non-finite value or one of magnitude >= 2^64");
    }
    std::vector<ReqView> reqs{R};
    s = run_requests(ctx, reqs, st);
    if (s == RRS_OK && !out_on_device) {
        CUDA_TRY(cudaMemcpyAsync(depth_out, R.depth_out, ob_depth, cudaMemcpyDeviceToHost, st));
        if (count_out) CUDA_TRY(cudaMemcpyAsync(count_out, R.count_out, ob_count, cudaMemcpyDeviceToHost, st));
        if (best_out) CUDA_TRY(cudaMemcpyAsync(best_out, R.best_out, ob_best, cudaMemcpyDeviceToHost, st));
        if (round_choice_out)
            CUDA_TRY(cudaMemcpyAsync(round_choice_out, R.choice_out, ob_choice, cudaMemcpyDeviceToHost, st));
    }
    if (zdev) cudaFreeAsync(zdev, st);
    if (outdev) cudaFreeAsync(outdev, st);
    if (s == RRS_OK && !out_on_device) s = check_device_errors(ctx, st);
    return s;
}

rrs_status rrs_depth_batched(rrs_ctx* ctx, const rrs_request* reqs, int32_t n_requests, int32_t use_graph,
                             void* stream)
{
    if (!ctx || (n_requests > 0 && !reqs) || n_requests < 0) return fail(RRS_ERR_INVALID_ARG, "bad arguments");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<ReqView> views;
    for (int i = 0; i < n_requests; ++i) {
        const rrs_request& q = reqs[i];
        rrs_status s = validate_params(q.kind, q.n_dirs, q.n_refinements, q.cap_shrink, q.dtype, q.precision);
        if (s != RRS_OK) {
            const std::string why = rrs_last_error();
            return fail(s, "request %d: %s", i, why.c_str());
        }
        if (q.n_queries < 0 || (q.n_queries > 0 && (!q.Z || !q.depth_out)))
            return fail(RRS_ERR_INVALID_ARG, "request %d: bad query batch or outputs", i);
        auto it = ctx->datasets.find(q.dataset_id);
        if (it == ctx->datasets.end()) return fail(RRS_ERR_NOT_FOUND, "request %d: no dataset %lld", i,
                                                   (long long)q.dataset_id);
        if (q.n_queries == 0) continue;
        if (q.precision == RRS_PREC_SPLIT_BF16X3) {
            s = ensure_bf16_planes(ctx, it->second);
            if (s != RRS_OK) return s;
        }
        ReqView R{};
        R.dset = &it->second;
        R.precision = q.precision;
        R.Z = q.Z;
        R.nq = q.n_queries;
        R.dtype = q.dtype;
        R.kind = q.kind;
        R.k = q.n_dirs;
        R.r = q.n_refinements;
        R.alpha = (float)q.cap_shrink;
        R.seed = q.seed;
        R.depth_out = q.depth_out;
        R.count_out = q.count_out;
        R.best_out = q.best_out;
        R.choice_out = q.round_choice_out;
        R.q_base = 0;
        views.push_back(R);
    }
    if (views.empty()) return RRS_OK;
    if (!use_graph) return run_requests(ctx, views, st);

    // graph path: identical descriptors replay a captured launch sequence
    std::vector<char> key((const char*)reqs, (const char*)reqs + sizeof(rrs_request) * n_requests);
    for (auto& g : ctx->graphs) {
        if (g.key == key) {
            CUDA_TRY(cudaGraphLaunch(g.exec, st));
            ctx->launches += g.launches;
            return RRS_OK;
        }
    }
    Plan P;
    P.tune = &ctx->pd_tune;
    P.tc_tune = &ctx->tc_tune;
    rrs_status s = build_plan(views, P);
    if (s != RRS_OK) return s;
    Carve sizing;
    const size_t bytes = carve_plan(P, sizing);
    if (!budget_ok(ctx, bytes)) return fail(RRS_ERR_BUDGET, "batched workspace needs %zu bytes", bytes);
    rrs_ctx::GraphEntry G;
    G.key = key;
    CUDA_TRY(cudaMalloc(&G.ws, bytes));
    G.ws_bytes = bytes;
    Carve C;
    C.base = (char*)G.ws;
    C.cap = bytes;
    carve_plan(P, C);
    s = upload_plan(ctx, P, st);
    if (s != RRS_OK) {
        cudaFree(G.ws);
        return s;
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    cudaStream_t cap;
    CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    const uint64_t before = ctx->launches;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        s = enqueue_rounds(ctx, P, cap, true);
        e = cudaStreamEndCapture(cap, &graph);
    }
    cudaStreamDestroy(cap);
    if (s != RRS_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaFree(G.ws);
        return s != RRS_OK ? s : fail(RRS_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    }
    G.launches = ctx->launches - before;
    e = cudaGraphInstantiate(&G.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaFree(G.ws);
        return fail(RRS_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    ctx->used += bytes;
    ctx->graphs.push_back(G);
    CUDA_TRY(cudaGraphLaunch(G.exec, st));
    return RRS_OK;
}

rrs_status rrs_debug_directions(rrs_ctx* ctx, uint64_t seed, int32_t q, int32_t round, int32_t m, int32_t d,
                                double cap_shrink, const float* pole, float* U)
{
    if (!ctx || !U || m < 0 || d < 1 || round < 1 || q < 0 || (round > 1 && !pole))
        return fail(RRS_ERR_INVALID_ARG, "bad arguments");
    CUDA_TRY(cudaSetDevice(ctx->device));
    const float* p = pole;
    float* tmp = nullptr;
    if (!p) {
        CUDA_TRY(cudaMalloc(&tmp, sizeof(float) * d));
        CUDA_TRY(cudaMemset(tmp, 0, sizeof(float) * d));
        p = tmp;
    }
    CUDA_TRY(launch_debug_dirs(seed, q, round - 1, m, d, (float)cap_shrink, p, U, 0));
    ctx->launches++;
    CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(tmp);
    return RRS_OK;
}

rrs_status rrs_debug_round_depths(rrs_ctx* ctx, int64_t dataset_id, const void* Z, int64_t n_queries, int32_t dtype,
                                  int32_t kind, int32_t m, const float* U, int32_t precision, double* depth_out,
                                  int64_t* count_out, int64_t* band_out)
{
    if (!ctx || !Z || !U || !depth_out || n_queries < 1 || m < 1) return fail(RRS_ERR_INVALID_ARG, "bad arguments");
    rrs_status s = validate_params(kind, m, 1, 0.5, dtype, precision);
    if (s != RRS_OK) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->datasets.find(dataset_id);
    if (it == ctx->datasets.end()) return fail(RRS_ERR_NOT_FOUND, "no dataset");
    CUDA_TRY(cudaSetDevice(ctx->device));
    Dataset& D = it->second;
    if (precision == RRS_PREC_SPLIT_BF16X3) {
        s = ensure_bf16_planes(ctx, D);
        if (s != RRS_OK) return s;
    }
    ReqView R{};
    R.dset = &D;
    R.Z = Z;
    R.nq = n_queries;
    R.dtype = dtype;
    R.kind = kind;
    R.k = m;
    R.r = 1;
    R.alpha = 0.5f;
    R.precision = precision;
    std::vector<ReqView> reqs{R};
    Plan P;
    s = build_plan(reqs, P);
    if (s != RRS_OK) return s;
    Carve sizing;
    const size_t bytes = carve_plan(P, sizing) + sizeof(int64_t) * n_queries + 512;
    void* ws = nullptr;
    CUDA_TRY(cudaMalloc(&ws, bytes));
    Carve C;
    C.base = (char*)ws;
    carve_plan(P, C);
    int64_t* band = C.take<int64_t>(n_queries);
    cudaStream_t st = 0;
    trace("debug_round_depths: workspace %zu bytes", bytes);
    s = upload_plan(ctx, P, st);
    if (s == RRS_OK) {
        trace("debug_round_depths: plan uploaded");
        cudaMemsetAsync(band, 0, sizeof(int64_t) * n_queries, st);
        CUDA_TRY(launch_prep(P.d_slots, (int)P.slots.size(), P.d_ds, P.z32, P.z64, P.poles, st));
        // caller's directions replace the generated ones; y_z from the FP64 query
        CUDA_TRY(launch_scatter_dirs(P.d_slots, (int)P.slots.size(), m, D.d, U, P.U, st));
        trace("debug_round_depths: directions scattered");
        CUDA_TRY(launch_yz_only(P.d_gen, (int)P.gen_tasks.size(), P.d_slots, P.z64, P.U, P.yz, st));
        trace("debug_round_depths: y_z done");
        if (kind == RRS_HALFSPACE) {
            if (precision == RRS_PREC_SPLIT_BF16X3)
                CUDA_TRY(launch_hd_tc(P.tc[0].d, (int)P.tc[0].tasks.size(), P.tc[0].kp, P.tc[0].bn, P.d_slots, P.d_ds, P.d_maps, P.U, P.yz,
                                      P.z64, P.res, band, ctx->d_err, st));
            else
                CUDA_TRY(launch_hd_simt(P.d_hd, (int)P.hd_tasks.size(), P.max_ldx, P.d_slots, P.d_ds, P.U, P.yz,
                                        P.z64, P.res, band, ctx->d_err, st));
        } else {
            for (size_t c = 0; c < P.pd_tasks.size(); ++c)
                if (!P.pd_tasks[c].empty())
                    CUDA_TRY(launch_pdap(P.d_pd[c], (int)P.pd_tasks[c].size(), P.pd_smem[c], P.pd_group[c],
                                         P.pd_variant[c], P.d_slots, P.d_ds, P.U,
                                         P.yz, P.res, ctx->d_err, st));
        }
        ctx->launches += 4;
        trace("debug_round_depths: depth kernels enqueued");
        std::vector<ResDev> hres(P.tot_m);
        CUDA_TRY(cudaMemcpyAsync(hres.data(), P.res, sizeof(ResDev) * P.tot_m, cudaMemcpyDeviceToHost, st));
        std::vector<int64_t> hband(n_queries);
        CUDA_TRY(cudaMemcpyAsync(hband.data(), band, sizeof(int64_t) * n_queries, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        trace("debug_round_depths: results copied");
        std::vector<double> dep(P.tot_m);
        std::vector<int64_t> cnt(P.tot_m);
        for (int64_t i = 0; i < P.tot_m; ++i) {
            dep[i] = hres[i].depth;
            cnt[i] = hres[i].count;
        }
        CUDA_TRY(cudaMemcpy(depth_out, dep.data(), sizeof(double) * P.tot_m, cudaMemcpyHostToDevice));
        if (count_out) CUDA_TRY(cudaMemcpy(count_out, cnt.data(), sizeof(int64_t) * P.tot_m, cudaMemcpyHostToDevice));
        if (band_out) CUDA_TRY(cudaMemcpy(band_out, hband.data(), sizeof(int64_t) * n_queries, cudaMemcpyHostToDevice));
        s = check_device_errors(ctx, st);
    }
    cudaFree(ws);
    return s;
}

rrs_status rrs_debug_wait_timeout(rrs_ctx* ctx, int64_t limit_cycles)
{
    if (!ctx || limit_cycles < 0) return fail(RRS_ERR_INVALID_ARG, "bad arguments");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(cudaMemset(ctx->d_err, 0, sizeof(int)));
    CUDA_TRY(launch_wait_probe(ctx->d_err, (long long)limit_cycles, 0));
    ctx->launches++;
    int h = 0;
    CUDA_TRY(cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(ctx->d_err, 0, sizeof(int)));
    if (h & ERR_TIMEOUT) return fail(RRS_ERR_TIMEOUT, "bounded device wait gave up after %lld cycles",
                                     (long long)limit_cycles);
    return RRS_OK;
}

rrs_status rrs_autotune(rrs_ctx* ctx, int64_t dataset_id, int32_t kind, int32_t n_dirs, int32_t n_refinements,
                        int32_t* choice_out)
{
    if (!ctx) return fail(RRS_ERR_INVALID_ARG, "NULL context");
    rrs_status s = validate_params(kind, n_dirs, n_refinements, 0.5, RRS_F32, RRS_PREC_FP32_SIMT);
    if (s != RRS_OK) return s;
    if (choice_out) *choice_out = 0;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->datasets.find(dataset_id);
    if (it == ctx->datasets.end()) return fail(RRS_ERR_NOT_FOUND, "no dataset %lld", (long long)dataset_id);
    CUDA_TRY(cudaSetDevice(ctx->device));
    Dataset& D = it->second;
    // halfspace: the tensor-core tile width where two exist (planes of K extent 64); the FP32 path has
    // nothing to tune
    if (kind == RRS_HALFSPACE && (!hd_tc_supported(D.d) || (int)align_up(D.d + 2, 64) != 64)) {
        if (choice_out && hd_tc_supported(D.d)) *choice_out = tc_tile_n((int)align_up(D.d + 2, 64));
        return RRS_OK;
    }
    if (kind == RRS_HALFSPACE) {
        s = ensure_bf16_planes(ctx, D);
        if (s != RRS_OK) return s;
    }
    const int m = (n_dirs + n_refinements - 1) / n_refinements;
    const auto key = std::make_tuple(D.n, D.ldx, m);
    // probe queries: the first rows of the data cloud, 2 per SM
    int nsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    const int64_t nq = std::min<int64_t>(D.n, 2 * (int64_t)nsm);
    std::vector<float> rows((size_t)nq * D.ldx), zh((size_t)nq * D.d);
    CUDA_TRY(cudaMemcpy(rows.data(), D.X32, sizeof(float) * rows.size(), cudaMemcpyDeviceToHost));
    for (int64_t q = 0; q < nq; ++q)
        for (int l = 0; l < D.d; ++l) zh[(size_t)q * D.d + l] = rows[(size_t)q * D.ldx + l];
    float* zd = nullptr;
    CUDA_TRY(cudaMalloc(&zd, sizeof(float) * zh.size()));
    CUDA_TRY(cudaMemcpy(zd, zh.data(), sizeof(float) * zh.size(), cudaMemcpyHostToDevice));
    double* dep = nullptr;
    CUDA_TRY(cudaMalloc(&dep, sizeof(double) * nq));
    cudaEvent_t a, b;
    CUDA_TRY(cudaEventCreate(&a));
    CUDA_TRY(cudaEventCreate(&b));
    int best = 0;
    float best_ms = 0.0f;
    const bool hd = kind == RRS_HALFSPACE;
    const auto tc_key = std::make_pair(D.n, 64);
    const std::vector<int> cands = hd ? std::vector<int>{256, 128}
                                      : std::vector<int>{1, 2, 4, PDAP_WARP_GROUP, PDAP_STREAM_CHOICE};
    for (int G : cands) {
        if (!hd && (G == PDAP_WARP_GROUP ? !pdapw_eligible(D.n, D.d)
                                         : (G != PDAP_STREAM_CHOICE &&
                                            (G > m || pdap_smem_bytes((int)D.n, G, D.ldx) > pdap_smem_limit()))))
            continue;
        if (hd) ctx->tc_tune[tc_key] = G;
        ReqView R{};
        R.dset = &D;
        R.Z = zd;
        R.nq = nq;
        R.dtype = RRS_F32;
        R.kind = kind;
        R.k = m;
        R.r = 1;
        R.alpha = 0.5f;
        R.depth_out = dep;
        if (hd) R.precision = RRS_PREC_SPLIT_BF16X3;
        float t = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            std::vector<ReqView> reqs{R};
            CUDA_TRY(cudaEventRecord(a, 0));
            s = run_requests(ctx, reqs, 0, hd ? 0 : G);
            if (s != RRS_OK) break;
            CUDA_TRY(cudaEventRecord(b, 0));
            CUDA_TRY(cudaEventSynchronize(b));
            float ms = 0.0f;
            CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
            if (rep > 0) t = std::min(t, ms);   // first repetition warms up
        }
        if (s != RRS_OK) break;
        if (!best || t < best_ms) {
            best = G;
            best_ms = t;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(zd);
    cudaFree(dep);
    if (hd) ctx->tc_tune.erase(tc_key);
    if (s != RRS_OK) return s;
    if (best) {
        if (hd)
            ctx->tc_tune[tc_key] = best;
        else
            ctx->pd_tune[key] = best;
    }
    drop_graphs(ctx);
    if (choice_out) *choice_out = best;
    return check_device_errors(ctx, 0);
}

rrs_status rrs_select_kernel(rrs_ctx* ctx, int64_t dataset_id, int32_t n_dirs, int32_t n_refinements, int32_t choice)
{
    if (!ctx) return fail(RRS_ERR_INVALID_ARG, "NULL context");
    if (choice != 0 && choice != 1 && choice != 2 && choice != 4 && choice != PDAP_WARP_GROUP &&
        choice != PDAP_STREAM_CHOICE)
        return fail(RRS_ERR_INVALID_ARG, "unknown selection kernel choice %d", choice);
    if (n_refinements < 1 || n_dirs < n_refinements) return fail(RRS_ERR_INVALID_ARG, "need n_dirs >= n_refinements >= 1");
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->datasets.find(dataset_id);
    if (it == ctx->datasets.end()) return fail(RRS_ERR_NOT_FOUND, "no dataset %lld", (long long)dataset_id);
    const Dataset& D = it->second;
    const int m = (int)(((int64_t)n_dirs + n_refinements - 1) / n_refinements);
    const auto key = std::make_tuple(D.n, D.ldx, m);
    if (choice == 0)
        ctx->pd_tune.erase(key);
    else
        ctx->pd_tune[key] = choice;
    drop_graphs(ctx);
    return RRS_OK;
}

rrs_status rrs_select_tc_tile(rrs_ctx* ctx, int64_t dataset_id, int32_t tile_points)
{
    if (!ctx) return fail(RRS_ERR_INVALID_ARG, "NULL context");
    if (tile_points != 0 && tile_points != 128 && tile_points != 256)
        return fail(RRS_ERR_INVALID_ARG, "tile width %d: 0, 128 or 256", tile_points);
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->datasets.find(dataset_id);
    if (it == ctx->datasets.end()) return fail(RRS_ERR_NOT_FOUND, "no dataset %lld", (long long)dataset_id);
    const Dataset& D = it->second;
    if (!hd_tc_supported(D.d)) return fail(RRS_ERR_UNSUPPORTED, "d=%d has no tensor-core path", D.d);
    const int kp = (D.d + 2 + 63) / 64 * 64;
    const auto key = std::make_pair(D.n, kp);
    if (tile_points == 0)
        ctx->tc_tune.erase(key);
    else
        ctx->tc_tune[key] = tile_points;
    drop_graphs(ctx);
    return RRS_OK;
}

rrs_status rrs_check(rrs_ctx* ctx, void* stream)
{
    if (!ctx) return fail(RRS_ERR_INVALID_ARG, "NULL context");
    CUDA_TRY(cudaSetDevice(ctx->device));
    return check_device_errors(ctx, (cudaStream_t)stream);
}

uint64_t rrs_launch_count(rrs_ctx* ctx) { return ctx ? ctx->launches : 0; }

rrs_status rrs_profile_enable(rrs_ctx* ctx, int32_t on)
{
    if (!ctx) return fail(RRS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->profiling = on != 0;
    for (int i = 0; i < RRS_NSTAGES; ++i) {
        ctx->stage_ms[i] = 0.0;
        ctx->stage_launches[i] = 0;
    }
    return RRS_OK;
}

rrs_status rrs_profile_read(rrs_ctx* ctx, double* ms_out, int64_t* launches_out)
{
    if (!ctx || !ms_out) return fail(RRS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    for (auto& m : ctx->marks) {
        CUDA_TRY(cudaEventSynchronize(m.b));
        float ms = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&ms, m.a, m.b));
        ctx->stage_ms[m.stage] += ms;
        ctx->event_pool.push_back(m.a);
        ctx->event_pool.push_back(m.b);
    }
    ctx->marks.clear();
    for (int i = 0; i < RRS_NSTAGES; ++i) {
        ms_out[i] = ctx->stage_ms[i];
        if (launches_out) launches_out[i] = ctx->stage_launches[i];
    }
    return RRS_OK;
}

}  // extern "C"
