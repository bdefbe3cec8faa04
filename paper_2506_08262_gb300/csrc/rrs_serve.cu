// Serving loop: continuous (iteration-level) batching of RRS depth requests.
//
// A server owns a fixed pool of query slots on the device.  Requests wait in a
// FIFO until enough slots are free; every rrs_server_step admits what fits,
// then runs ONE refinement round (Alg. 4: generate, project + univariate depth,
// minimum and pole update) for a set of admitted queries in shared launches --
// each query (slot) at its own round -- and retires the requests whose queries
// have all run their last round, copying their depths to the caller's host
// buffer.  The set is bounded by a work limit (weighted point-direction pairs
// per step): every admitted request, oldest first, may take up to a quarter of
// the limit (at least one query), then the oldest requests fill the rest.  So
// a step's duration stays bounded however much is admitted, small requests
// progress beside large ones, and a large request runs its queries in pieces
// at full occupancy.  A request joins the GPU work of requests already in
// flight at the next step, and its results do not depend on what else is in
// the mix: every query keeps its own direction stream (counter index = row
// within its request) and state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <tuple>
#include <vector>

#include "../../include/rrs.h"
#include "rrs_ctx.h"
#include "rrs_internal.h"

using namespace rrs;

namespace {

rrs_status sfail(rrs_status st, const char* fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    set_last_error(msg);
    return st;
}

#define S_TRY(expr)                                                                                  \
    do {                                                                                             \
        cudaError_t _e = (expr);                                                                     \
        if (_e != cudaSuccess) {                                                                     \
            cudaGetLastError();                                                                      \
            return sfail(RRS_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e));                     \
        }                                                                                            \
    } while (0)

struct Request {
    int64_t id;
    int64_t dataset;
    const void* Zhost;
    int64_t nq;
    int32_t dtype, kind, k, r, m;
    float alpha;
    uint64_t seed;
    double* out_host;
    // device side once admitted
    void* zdev = nullptr;
    double* ddev = nullptr;
    std::vector<int32_t> slots;
    std::vector<int32_t> sround;   // rounds run by each of its slots
    int64_t rounds_left = 0;       // sum over its slots of the rounds still to run
    double slot_work = 0.0;        // weighted point-direction pairs of one round of one query
    cudaEvent_t done = nullptr;
    bool finished = false;
};

// Admit kernel: place the new slots' descriptors and prepare their state.
__global__ void k_admit(const SlotDev* __restrict__ src, const int32_t* __restrict__ idx, int cnt,
                        SlotDev* __restrict__ slots, const DsDev* __restrict__ ds, float* __restrict__ z32,
                        double* __restrict__ z64, float* __restrict__ poles0)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    SlotDev S = src[t];
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
        poles0[S.zoff32 + l] = (l == 0) ? 1.0f : 0.0f;
    }
    S.znorm = __double2float_ru(__dsqrt_ru(acc) * (1.0 + 1e-12));
    S.dmin = 1.0;
    S.cmin = ds[S.ds].n;
    S.best = -1;
    S.round = 0;
    slots[idx[t]] = S;
}

}  // namespace

struct rrs_server {
    rrs_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    int cap = 0, max_m = 0, max_d = 0, max_ldx = 0;
    int precision = RRS_PREC_FP32_SIMT;   // halfspace arithmetic (tensor cores where the dataset allows)
    // device arena
    void* arena = nullptr;
    size_t arena_bytes = 0;
    SlotDev* d_slots = nullptr;
    float *d_z32 = nullptr, *d_p0 = nullptr, *d_p1 = nullptr, *d_U = nullptr;
    double *d_z64 = nullptr, *d_yz = nullptr;
    ResDev* d_res = nullptr;
    DsDev* d_ds = nullptr;
    CUtensorMap* d_maps = nullptr;   // tensor map of each dataset row with BF16 planes (tensor-core halfspace)
    int ds_cap = 0;
    char* d_tab = nullptr;      // per-step tables (tasks, lists, new slots)
    size_t tab_bytes = 0;
    float* d_keys = nullptr;    // selection keys formed by k_keys for d > 16 (at most KEYS_SCRATCH_BYTES)
    size_t keys_bytes = 0;
    // host
    std::vector<int32_t> free_slots;
    std::deque<Request*> pending;
    std::map<int64_t, Request*> requests;
    std::vector<Request*> active;
    std::map<int64_t, int> ds_index;   // dataset id -> row of d_ds
    std::vector<DsDev> ds_host;
    std::vector<int> ds_bn;            // tensor-core tile width of each dataset row (0: no planes)
    int64_t next_id = 1;
    int active_queries = 0;
    double work_limit = RRS_SERVER_DEFAULT_WORK;   // weighted pairs per step (0: every admitted query)
};

namespace {

int padded(int d)
{
    int l = (d + 3) & ~3;
    if (((l / 4) & 1) == 0) l += 4;
    return l;
}

rrs_status ensure_dataset(rrs_server* S, int64_t id, int* row)
{
    auto f = S->ds_index.find(id);
    if (f != S->ds_index.end()) {
        *row = f->second;
        return RRS_OK;
    }
    auto it = S->ctx->datasets.find(id);
    if (it == S->ctx->datasets.end()) return sfail(RRS_ERR_NOT_FOUND, "no dataset %lld", (long long)id);
    if ((int)S->ds_host.size() >= S->ds_cap) return sfail(RRS_ERR_BUDGET, "server dataset table full");
    Dataset& D = it->second;
    if (S->precision == RRS_PREC_SPLIT_BF16X3 && hd_tc_supported(D.d)) {
        const rrs_status s = ensure_bf16_planes(S->ctx, D);
        if (s != RRS_OK) return s;
    }
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
    const int r = (int)S->ds_host.size();
    S->ds_host.push_back(dd);
    S_TRY(cudaMemcpyAsync(S->d_ds + r, &S->ds_host[r], sizeof(DsDev), cudaMemcpyHostToDevice, S->st));
    int bn = 0;
    if (dd.Xbf) {
        auto t = S->ctx->tc_tune.find(std::make_pair(dd.n, dd.kp));
        bn = tc_tile_n(dd.kp, t == S->ctx->tc_tune.end() ? 0 : t->second);
        CUtensorMap map;
        S_TRY(encode_tc_map(dd, bn, &map));
        S_TRY(cudaMemcpyAsync(S->d_maps + r, &map, sizeof map, cudaMemcpyHostToDevice, S->st));
        S_TRY(cudaStreamSynchronize(S->st));   // the host copy of the map goes out of scope here
    }
    S->ds_index[id] = r;
    S->ds_bn.push_back(bn);
    *row = r;
    return RRS_OK;
}

// Carve one per-step table area, growing it (stream-ordered) when needed.
rrs_status step_table(rrs_server* S, size_t bytes)
{
    if (bytes <= S->tab_bytes) return RRS_OK;
    if (S->d_tab) S_TRY(cudaFreeAsync(S->d_tab, S->st));
    const size_t nb = std::max(bytes, S->tab_bytes * 2);
    S_TRY(cudaMallocAsync((void**)&S->d_tab, nb, S->st));
    S->tab_bytes = nb;
    return RRS_OK;
}

rrs_status admit(rrs_server* S)
{
    std::vector<SlotDev> news;
    std::vector<int32_t> idx;
    while (!S->pending.empty()) {
        Request* R = S->pending.front();
        if ((int64_t)S->free_slots.size() < R->nq) break;
        int row = 0;
        rrs_status s = ensure_dataset(S, R->dataset, &row);
        if (s != RRS_OK) return s;
        const DsDev& D = S->ds_host[row];
        const size_t esz = R->dtype == RRS_F32 ? 4 : 8;
        const size_t zbytes = esz * (size_t)R->nq * D.d;
        S_TRY(cudaMallocAsync(&R->zdev, zbytes, S->st));
        S_TRY(cudaMallocAsync((void**)&R->ddev, sizeof(double) * R->nq, S->st));
        S_TRY(cudaMemcpyAsync(R->zdev, R->Zhost, zbytes, cudaMemcpyHostToDevice, S->st));
        // cost weight of a pair: the tensor-core halfspace path runs about ten times as many pairs per second
        // as the FP32 and selection paths (measured)
        const bool tc = R->kind == RRS_HALFSPACE && S->precision == RRS_PREC_SPLIT_BF16X3 && D.kp > 0;
        R->slot_work = (double)D.n * R->m * (tc ? 0.1 : 1.0);
        R->sround.assign((size_t)R->nq, 0);
        R->rounds_left = R->nq * (int64_t)R->r;
        for (int64_t q = 0; q < R->nq; ++q) {
            const int32_t slot = S->free_slots.back();
            S->free_slots.pop_back();
            R->slots.push_back(slot);
            SlotDev sd{};
            sd.ds = row;
            sd.kind = R->kind;
            sd.m = R->m;
            sd.r = R->r;
            sd.alpha = R->alpha;
            sd.d = D.d;
            sd.ldx = D.ldx;
            sd.zdtype = R->dtype;
            sd.seed = R->seed;
            sd.qctr = q;
            sd.uoff = (int64_t)slot * S->max_m * S->max_ldx;
            sd.roff = (int64_t)slot * S->max_m;
            sd.zoff32 = (int64_t)slot * S->max_ldx;
            sd.zoff64 = (int64_t)slot * S->max_d;
            sd.zsrc = (const char*)R->zdev + (size_t)q * D.d * esz;
            sd.depth_out = R->ddev + q;
            news.push_back(sd);
            idx.push_back(slot);
        }
        S->pending.pop_front();
        S->active.push_back(R);
        S->active_queries += (int)R->nq;
    }
    if (news.empty()) return RRS_OK;
    const size_t b1 = sizeof(SlotDev) * news.size(), b2 = sizeof(int32_t) * idx.size();
    char* tmp = nullptr;
    S_TRY(cudaMallocAsync((void**)&tmp, b1 + 256 + b2, S->st));
    S_TRY(cudaMemcpyAsync(tmp, news.data(), b1, cudaMemcpyHostToDevice, S->st));
    S_TRY(cudaMemcpyAsync(tmp + b1 + 256 - (b1 % 256), idx.data(), b2, cudaMemcpyHostToDevice, S->st));
    const int cnt = (int)news.size();
    k_admit<<<(cnt + 127) / 128, 128, 0, S->st>>>((const SlotDev*)tmp, (const int32_t*)(tmp + b1 + 256 - (b1 % 256)),
                                                 cnt, S->d_slots, S->d_ds, S->d_z32, S->d_z64, S->d_p0);
    S_TRY(cudaGetLastError());
    S->ctx->launches++;
    S_TRY(cudaFreeAsync(tmp, S->st));
    return RRS_OK;
}

}  // namespace

extern "C" {

rrs_status rrs_server_create(rrs_ctx* ctx, int32_t max_slots, int32_t max_dirs_per_round, int32_t max_d,
                             int32_t precision, void* stream, rrs_server** out)
{
    if (!ctx || !out || max_slots < 1 || max_dirs_per_round < 1 || max_d < 1 || max_d > 1024 ||
        (precision != RRS_PREC_FP32_SIMT && precision != RRS_PREC_SPLIT_BF16X3))
        return sfail(RRS_ERR_INVALID_ARG, "bad server parameters");
    *out = nullptr;
    std::lock_guard<std::mutex> lk(ctx->mu);
    S_TRY(cudaSetDevice(ctx->device));
    rrs_server* S = new rrs_server;
    S->ctx = ctx;
    S->st = (cudaStream_t)stream;
    S->cap = max_slots;
    S->max_m = max_dirs_per_round;
    S->max_d = max_d;
    S->max_ldx = padded(max_d);
    S->precision = precision;
    S->ds_cap = 4096;
    const size_t c = (size_t)max_slots;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return at;
    };
    const size_t o_slots = take(sizeof(SlotDev) * c), o_z32 = take(sizeof(float) * c * S->max_ldx),
                 o_p0 = take(sizeof(float) * c * S->max_ldx), o_p1 = take(sizeof(float) * c * S->max_ldx),
                 o_z64 = take(sizeof(double) * c * max_d), o_U = take(sizeof(float) * c * S->max_m * S->max_ldx),
                 o_yz = take(sizeof(double) * c * S->max_m), o_res = take(sizeof(ResDev) * c * S->max_m),
                 o_ds = take(sizeof(DsDev) * S->ds_cap), o_maps = take(sizeof(CUtensorMap) * S->ds_cap);
    if (ctx->budget && ctx->used + off > ctx->budget) {
        delete S;
        return sfail(RRS_ERR_BUDGET, "server arena needs %zu bytes", off);
    }
    cudaError_t e = cudaMalloc(&S->arena, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return sfail(RRS_ERR_CUDA, "server arena: %s", cudaGetErrorString(e));
    }
    ctx->used += off;
    S->arena_bytes = off;
    char* B = (char*)S->arena;
    S->d_slots = (SlotDev*)(B + o_slots);
    S->d_z32 = (float*)(B + o_z32);
    S->d_p0 = (float*)(B + o_p0);
    S->d_p1 = (float*)(B + o_p1);
    S->d_z64 = (double*)(B + o_z64);
    S->d_U = (float*)(B + o_U);
    S->d_yz = (double*)(B + o_yz);
    S->d_res = (ResDev*)(B + o_res);
    S->d_ds = (DsDev*)(B + o_ds);
    S->d_maps = (CUtensorMap*)(B + o_maps);
    for (int i = max_slots - 1; i >= 0; --i) S->free_slots.push_back(i);
    *out = S;
    return RRS_OK;
}

rrs_status rrs_server_submit(rrs_server* S, int64_t dataset_id, const void* Z, int64_t n_queries, int32_t dtype,
                             int32_t kind, int32_t n_dirs, int32_t n_refinements, double cap_shrink, uint64_t seed,
                             double* depth_out, int64_t* request_id_out)
{
    if (!S || !request_id_out || n_queries < 1 || !Z || !depth_out) return sfail(RRS_ERR_INVALID_ARG, "bad request");
    if (kind < 0 || kind > 2 || n_refinements < 1 || n_dirs < n_refinements || !(cap_shrink > 0.0) ||
        cap_shrink > 1.0 || (dtype != RRS_F32 && dtype != RRS_F64))
        return sfail(RRS_ERR_INVALID_ARG, "bad request parameters");
    std::lock_guard<std::mutex> lk(S->ctx->mu);
    auto it = S->ctx->datasets.find(dataset_id);
    if (it == S->ctx->datasets.end()) return sfail(RRS_ERR_NOT_FOUND, "no dataset %lld", (long long)dataset_id);
    const int m = (n_dirs + n_refinements - 1) / n_refinements;
    if (m > S->max_m || it->second.d > S->max_d || n_queries > S->cap)
        return sfail(RRS_ERR_UNSUPPORTED, "request exceeds the server's slot shape (m=%d, d=%d, nq=%lld)", m,
                     it->second.d, (long long)n_queries);
    if (kind != RRS_HALFSPACE && it->second.n > PDAP_MAX_N)
        return sfail(RRS_ERR_UNSUPPORTED, "n too large for the selection kernel");
    Request* R = new Request;
    R->id = S->next_id++;
    R->dataset = dataset_id;
    R->Zhost = Z;
    R->nq = n_queries;
    R->dtype = dtype;
    R->kind = kind;
    R->k = n_dirs;
    R->r = n_refinements;
    R->m = m;
    R->alpha = (float)cap_shrink;
    R->seed = seed;
    R->out_host = depth_out;
    S->pending.push_back(R);
    S->requests[R->id] = R;
    *request_id_out = R->id;
    return RRS_OK;
}

rrs_status rrs_server_step(rrs_server* S, int32_t* active_queries_out, int32_t* pending_requests_out)
{
    if (!S) return sfail(RRS_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(S->ctx->mu);
    S_TRY(cudaSetDevice(S->ctx->device));
    rrs_status s = admit(S);
    if (s != RRS_OK) return s;
    if (!S->active.empty()) {
        // queries of this step: every request, oldest first, up to a quarter of the work limit (at least one
        // query); then the oldest requests fill the rest.  pick[i] lists slot positions of active[i].
        const size_t na = S->active.size();
        std::vector<std::vector<int32_t>> pick(na);
        std::vector<size_t> cursor(na, 0);   // next slot position to consider
        const bool capped = S->work_limit > 0.0;
        double used = 0.0;
        auto take = [&](size_t i, double share) {
            Request* R = S->active[i];
            double mine = 0.0;
            while (cursor[i] < R->slots.size()) {
                const size_t p = cursor[i];
                if (R->sround[p] >= R->r) {
                    ++cursor[i];
                    continue;
                }
                const bool first = pick[i].empty() && (used == 0.0 || share < 1.0);
                if (capped && !first && (mine + R->slot_work > share * S->work_limit ||
                                         used + R->slot_work > S->work_limit))
                    break;
                pick[i].push_back((int32_t)p);
                mine += R->slot_work;
                used += R->slot_work;
                ++cursor[i];
            }
        };
        for (size_t i = 0; i < na; ++i) {
            if (capped && used >= S->work_limit) break;
            take(i, 0.25);
        }
        for (size_t i = 0; i < na && capped && used < S->work_limit; ++i) take(i, 1.0);
        // tables of this step: gen tasks, halfspace tasks, selection tasks per launch key, argmin list
        std::vector<TaskDev> gen, hd;
        // (K extent of the planes, points per tile) -> tensor-core halfspace tasks
        std::map<std::pair<int, int>, std::vector<TaskDev>> tc;
        // selection lists per (shared-memory class, G, kernel variant, dataset row for keys by k_keys or -1);
        // each launch requests the largest shared-memory need of its list
        std::map<std::tuple<size_t, int, int, int>, std::vector<TaskDev>> pd;
        std::map<std::tuple<size_t, int, int, int>, size_t> pd_need;
        std::vector<int32_t> arg;
        const size_t classes[] = {24 * 1024, 48 * 1024, 72 * 1024, 110 * 1024, pdap_smem_limit()};
        for (size_t ai = 0; ai < na; ++ai) {
            Request* R = S->active[ai];
            if (pick[ai].empty()) continue;
            const DsDev& D = S->ds_host[S->ds_index[R->dataset]];
            PdapShape sh{};
            size_t cls = 0;
            if (R->kind != RRS_HALFSPACE) {
                sh = pdap_shape((int)D.n, D.ldx, R->m, D.d);
                for (size_t c : classes)
                    if (sh.smem <= c) {
                        cls = c;
                        break;
                    }
            }
            const int G = sh.group;
            const int hper = (R->m + ((R->m + 63) / 64) - 1) / ((R->m + 63) / 64);
            const int row = S->ds_index[R->dataset];
            const bool use_tc = R->kind == RRS_HALFSPACE && S->precision == RRS_PREC_SPLIT_BF16X3 && D.kp > 0;
            for (int32_t pos : pick[ai]) {
                const int32_t slot = R->slots[pos];
                for (int j0 = 0; j0 < R->m; j0 += 128) gen.push_back(TaskDev{slot, j0, std::min(128, R->m - j0), 0});
                if (use_tc) {
                    // slots of a request need not be adjacent: one task never crosses a slot
                    auto& v = tc[std::make_pair(D.kp, S->ds_bn[row])];
                    for (int j0 = 0; j0 < R->m; j0 += 128) v.push_back(TaskDev{slot, j0, std::min(128, R->m - j0), 0});
                } else if (R->kind == RRS_HALFSPACE) {
                    for (int j0 = 0; j0 < R->m; j0 += hper) hd.push_back(TaskDev{slot, j0, std::min(hper, R->m - j0), 0});
                } else {
                    const int keys_row = sh.keys_gemm ? row : -1;
                    const auto key = std::make_tuple(cls, G, sh.variant, keys_row);
                    auto& v = pd[key];
                    size_t& need = pd_need[key];
                    need = std::max(need, sh.smem);
                    for (int j0 = 0; j0 < R->m; j0 += G) v.push_back(TaskDev{slot, j0, std::min(G, R->m - j0), row});
                }
                arg.push_back(slot);
            }
        }
        size_t need = sizeof(TaskDev) * (gen.size() + hd.size()) + sizeof(int32_t) * arg.size() + 1024;
        for (auto& kv : tc) need += sizeof(TaskDev) * kv.second.size() + 256;
        for (auto& kv : pd) need += sizeof(TaskDev) * kv.second.size() + 256;
        s = step_table(S, need);
        if (s != RRS_OK) return s;
        std::vector<char> host(need);
        size_t off = 0;
        auto put = [&](const void* p, size_t bytes) {
            const size_t at = off;
            memcpy(host.data() + off, p, bytes);
            off = (off + bytes + 255) & ~(size_t)255;
            return at;
        };
        const size_t o_gen = put(gen.data(), sizeof(TaskDev) * gen.size());
        const size_t o_hd = put(hd.data(), sizeof(TaskDev) * hd.size());
        const size_t o_arg = put(arg.data(), sizeof(int32_t) * arg.size());
        std::vector<std::pair<size_t, std::tuple<size_t, int, int, int>>> o_pd;
        for (auto& kv : pd) o_pd.push_back({put(kv.second.data(), sizeof(TaskDev) * kv.second.size()), kv.first});
        std::vector<std::pair<size_t, std::pair<int, int>>> o_tc;
        for (auto& kv : tc) o_tc.push_back({put(kv.second.data(), sizeof(TaskDev) * kv.second.size()), kv.first});
        S_TRY(cudaMemcpyAsync(S->d_tab, host.data(), off, cudaMemcpyHostToDevice, S->st));
        char* T = S->d_tab;
        S_TRY(launch_gen_slotround((const TaskDev*)(T + o_gen), (int)gen.size(), S->d_slots, S->d_p0, S->d_p1,
                                   S->d_z64, S->d_U, S->d_yz, S->max_ldx, S->st));
        S_TRY(launch_hd_simt((const TaskDev*)(T + o_hd), (int)hd.size(), S->max_ldx, S->d_slots, S->d_ds, S->d_U,
                             S->d_yz, S->d_z64, S->d_res, nullptr, S->ctx->d_err, S->st));
        for (auto& to : o_tc)
            S_TRY(launch_hd_tc((const TaskDev*)(T + to.first), (int)tc[to.second].size(), to.second.first,
                               to.second.second, S->d_slots, S->d_ds, S->d_maps, S->d_U, S->d_yz, S->d_z64, S->d_res,
                               nullptr, S->ctx->d_err, S->st));
        size_t extra = 0;
        for (auto& po : o_pd) {
            const auto& key = po.second;
            const TaskDev* tl = (const TaskDev*)(T + po.first);
            const int cnt_all = (int)pd[key].size(), G = std::get<1>(key), krow = std::get<3>(key);
            if (krow < 0) {
                S_TRY(launch_pdap(tl, cnt_all, pd_need[key], G, std::get<2>(key), S->d_slots, S->d_ds, S->d_U,
                                  S->d_yz, S->d_res, S->ctx->d_err, S->st));
                continue;
            }
            // d > 16: keys by the tiled GEMM, then the selection on them, one scratch-sized chunk at a time
            constexpr size_t KEYS_SCRATCH_BYTES = 256u << 20;
            const int n = (int)S->ds_host[krow].n;
            const size_t per = pdap_keys_bytes(n, G, 1);
            const int chunk = (int)std::max<size_t>(1, std::min<size_t>(cnt_all, KEYS_SCRATCH_BYTES / per));
            const size_t need_b = pdap_keys_bytes(n, G, chunk);
            if (need_b > S->keys_bytes) {
                if (S->d_keys) S_TRY(cudaFreeAsync(S->d_keys, S->st));
                S->d_keys = nullptr;
                S_TRY(cudaMallocAsync((void**)&S->d_keys, need_b, S->st));
                S->keys_bytes = need_b;
            }
            for (int t0 = 0; t0 < cnt_all; t0 += chunk) {
                const int cnt = std::min(chunk, cnt_all - t0);
                S_TRY(launch_pdap_keys(tl + t0, cnt, G, S->d_slots, S->d_ds, S->ds_host[krow], S->d_U, S->d_keys,
                                       S->st));
                S_TRY(launch_pdap(tl + t0, cnt, pd_need[key], G, std::get<2>(key), S->d_slots, S->d_ds, S->d_U,
                                  S->d_yz, S->d_res, S->ctx->d_err, S->st, S->d_keys));
                extra += 1 + PDAP_LAUNCH_KERNELS;
            }
            extra -= PDAP_LAUNCH_KERNELS;   // counted once below
        }
        S_TRY(launch_argmin_slotround(S->d_slots, (const int32_t*)(T + o_arg), (int)arg.size(), S->d_U, S->d_res,
                                     S->d_p0, S->d_p1, S->st));
        S->ctx->launches += 3 + pd.size() * PDAP_LAUNCH_KERNELS + tc.size() + extra;
        // retire requests whose last round just ran
        std::vector<Request*> still;
        for (size_t ai = 0; ai < na; ++ai) {
            for (int32_t pos : pick[ai]) S->active[ai]->sround[pos]++;
            S->active[ai]->rounds_left -= (int64_t)pick[ai].size();
        }
        for (Request* R : S->active) {
            if (R->rounds_left == 0) {
                S_TRY(cudaMemcpyAsync(R->out_host, R->ddev, sizeof(double) * R->nq, cudaMemcpyDeviceToHost, S->st));
                S_TRY(cudaEventCreateWithFlags(&R->done, cudaEventDisableTiming));
                S_TRY(cudaEventRecord(R->done, S->st));
                S_TRY(cudaFreeAsync(R->zdev, S->st));
                S_TRY(cudaFreeAsync(R->ddev, S->st));
                R->zdev = nullptr;
                R->ddev = nullptr;
                for (int32_t slot : R->slots) S->free_slots.push_back(slot);
                S->active_queries -= (int)R->nq;
                R->finished = true;
            } else {
                still.push_back(R);
            }
        }
        S->active.swap(still);
    }
    if (active_queries_out) *active_queries_out = S->active_queries;
    if (pending_requests_out) *pending_requests_out = (int32_t)S->pending.size();
    return RRS_OK;
}

rrs_status rrs_server_set_work_limit(rrs_server* S, double max_pairs_per_step)
{
    if (!S || !(max_pairs_per_step >= 0.0) || !(max_pairs_per_step <= 1e300))
        return sfail(RRS_ERR_INVALID_ARG, "bad work limit");
    std::lock_guard<std::mutex> lk(S->ctx->mu);
    S->work_limit = max_pairs_per_step;
    return RRS_OK;
}

rrs_status rrs_server_poll(rrs_server* S, int64_t request_id, int32_t* done_out)
{
    if (!S || !done_out) return sfail(RRS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->ctx->mu);
    auto it = S->requests.find(request_id);
    if (it == S->requests.end()) return sfail(RRS_ERR_NOT_FOUND, "no request %lld", (long long)request_id);
    Request* R = it->second;
    *done_out = 0;
    if (!R->finished) return RRS_OK;
    const cudaError_t e = cudaEventQuery(R->done);
    if (e == cudaErrorNotReady) return RRS_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(RRS_ERR_CUDA, "request event: %s", cudaGetErrorString(e));
    }
    cudaEventDestroy(R->done);
    S->requests.erase(it);
    delete R;
    *done_out = 1;
    return RRS_OK;
}

rrs_status rrs_server_destroy(rrs_server* S)
{
    if (!S) return RRS_OK;
    std::lock_guard<std::mutex> lk(S->ctx->mu);
    cudaSetDevice(S->ctx->device);
    cudaStreamSynchronize(S->st);
    for (auto& kv : S->requests) {
        Request* R = kv.second;
        if (R->zdev) cudaFree(R->zdev);
        if (R->ddev) cudaFree(R->ddev);
        if (R->done) cudaEventDestroy(R->done);
        delete R;
    }
    if (S->d_tab) cudaFree(S->d_tab);
    if (S->d_keys) cudaFree(S->d_keys);
    cudaFree(S->arena);
    S->ctx->used -= S->arena_bytes;
    delete S;
    return RRS_OK;
}

}  // extern "C"
