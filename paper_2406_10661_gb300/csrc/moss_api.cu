// Host side of the C ABI declared in include/moss.h: input validation, the
// union network of a batch, device buffers, CUDA-graph replay of the step
// kernels, and state / metric transfer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "moss.h"
#include "moss_kernels.cuh"

using namespace moss;

constexpr int RB_WORDS = M_NFIELDS + 2;  // readback slot: metric record, step, error word

namespace {

struct SnapBufs {
    void* a;     // RecA<Real>[cap]
    RecB* b;     // [cap]
    int32_t* off;
};

constexpr int N_STEP_KERNELS = 4;  // decide, resolve, lanescan, place (launch order)

}  // namespace

struct MossHandle {
    int precision = 32;
    int n_scen = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int sm_count = 1;
    MossParams prm{};
    std::string err;

    // ---- host copies of the (union) inputs
    int n_lanes = 0, n_junctions = 0, n_veh = 0, n_phases = 0;
    std::vector<LaneInfo> lanes;
    std::vector<int32_t> lane_src_road;  // junction lanes: the road they leave
    std::vector<int32_t> junc_scen, junc_phase_off;
    std::vector<int32_t> routes, dep, start_lane, veh_scen;
    std::vector<int2> route_span;     // route of vehicle g: routes[span.x .. span.y)
    size_t routes_cap = 0;            // capacity of d_routes (entries)
    int32_t* d_req = nullptr;         // [n_veh] re-routing marks (-1)
    std::vector<float> v0f;
    std::vector<int32_t> q_off, q_ids, start_lanes;
    std::vector<int32_t> scen_veh_off, scen_lane_off, scen_junc_off;
    std::vector<uint32_t> key0, key1;

    // ---- device
    std::vector<std::pair<void*, size_t>> allocs;  // device buffers and their sizes
    MossAllocator allocator{};                       // caller's device allocator (alloc == NULL: cudaMalloc)
    size_t bytes = 0;
    LaneInfo* d_lane = nullptr;
    float* d_v0f = nullptr;
    JuncInfo* d_junc = nullptr;
    int32_t *d_phase_green = nullptr, *d_phase_amber = nullptr, *d_junc_policy = nullptr,
            *d_junc_manual = nullptr, *d_junc_state = nullptr;
    int4* d_mp = nullptr;  // max-pressure state per junction
    int32_t *d_jj_off = nullptr, *d_jj_lane = nullptr, *d_jj_from = nullptr, *d_mp_press = nullptr;
    int n_jj = 0;
    bool lane_groups = false;         // some road has a turn that not all of its lanes serve (R27)
    std::vector<int32_t> jl_plans;    // plan mask per lane (junction lanes; 0xff = every plan), R28
    int32_t* d_jl_plans = nullptr;
    int8_t* d_road_mark = nullptr;    // roads whose plan a setter changes
    int2* d_road_span = nullptr;      // (first, end) road lanes per road
    std::vector<int2> road_span;
    std::vector<int> scen_road_off;   // [n_scen+1]
    int32_t* d_lstage = nullptr;      // setter arguments for lanes (2 * n_lanes)
    void* d_mbuf = nullptr;           // metric output (max(n_lanes, n_roads) doubles)
    int2* d_route_span = nullptr;
    int32_t *d_routes = nullptr, *d_dep = nullptr, *d_vstatus = nullptr,
            *d_vflags = nullptr;
    int32_t *d_q_off = nullptr, *d_q_ids = nullptr, *d_q_head = nullptr, *d_start_lanes = nullptr;
    uint32_t *d_key0 = nullptr, *d_key1 = nullptr;
    int32_t* d_veh_base = nullptr;
    long long *d_step = nullptr, *d_metrics = nullptr;
    SnapBufs snap[2]{};
    int8_t* d_code = nullptr;
    void* d_stay = nullptr;  // SV<Real>[cap]
    void* d_ea = nullptr;    // RecA<Real>[cap]
    RecB* d_eb = nullptr;
    int32_t *d_enext = nullptr, *d_enter = nullptr, *d_leave = nullptr, *d_lbefore = nullptr,
            *d_tile_leave = nullptr, *d_tile_prefix = nullptr;
    unsigned long long *d_head = nullptr, *d_lane_tiles = nullptr;
    void* d_cands = nullptr;  // Cand<Real>[cap]
    unsigned long long* d_gap_head = nullptr;
    int n_lane_tiles = 0, max_slot_tiles = 0, n_junc_chunks = 0;
    Counters* d_cnt = nullptr;  // [2]: per parity; d_cnt[0].err holds the device error bits
    int32_t* d_stage = nullptr;          // setter staging (2 * n_junctions)
    int32_t* h_stage = nullptr;          // pinned host staging of setter arguments (2 * n_junctions)
    cudaEvent_t stage_free = nullptr;    // recorded after the last copy out of h_stage
    // pinned readback: per slot a metric record, its step and the error word;
    // slots [0, MOSS_METRIC_SLOTS) serve moss_metrics_enqueue/read, the last
    // one moss_get_metrics
    long long* h_rb = nullptr;
    cudaEvent_t rb_ev[MOSS_METRIC_SLOTS] = {};
    int rb_scen[MOSS_METRIC_SLOTS] = {};
    bool rb_pending[MOSS_METRIC_SLOTS] = {};

    // launch configuration (blocks per SM) of the step kernels; moss_autotune picks them
    int cfg_decide = MOSS_DECIDE_MIN_BLOCKS, cfg_lanescan = 4, cfg_place = 8;

    int parity = 0;  // snapshot buffer holding the current step
    cudaGraphExec_t g2[2] = {nullptr, nullptr}, g1[2] = {nullptr, nullptr};
    bool timing = false;
    cudaEvent_t ev[N_STEP_KERNELS + 1] = {};
    double kms[4] = {0, 0, 0, 0};
    long long ksteps = 0;
};

namespace {

int fail(MossHandle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

int cuda_fail(MossHandle* h, cudaError_t e, const char* what) {
    return fail(h, MOSS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);        \
    } while (0)

// device memory of the handle: the caller's allocator when one was given
// (on the handle's stream), else cudaMalloc; nullptr on failure
void* raw_alloc(MossHandle* h, size_t nb) {
    if (h->allocator.alloc) return h->allocator.alloc(nb, (void*)h->stream, h->allocator.ctx);
    void* q = nullptr;
    if (cudaMalloc(&q, nb) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return q;
}

void raw_free(MossHandle* h, void* p, size_t nb) {
    if (!p) return;
    if (h->allocator.alloc) h->allocator.release(p, nb, (void*)h->stream, h->allocator.ctx);
    else cudaFree(p);
}

template <typename T>
int dalloc(MossHandle* h, T** p, size_t count) {
    const size_t nb = std::max<size_t>(count, 1) * sizeof(T);
    void* q = raw_alloc(h, nb);
    if (!q) return fail(h, MOSS_ENOMEM, "device allocation of " + std::to_string(nb) + " bytes failed");
    h->allocs.emplace_back(q, nb);
    h->bytes += nb;
    *p = (T*)q;
    return MOSS_OK;
}

template <typename T>
int upload(MossHandle* h, T** p, const std::vector<T>& v) {
    int rc = dalloc(h, p, v.size());
    if (rc) return rc;
    if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    return MOSS_OK;
}

#define TRY(call)              \
    do {                       \
        int r_ = (call);       \
        if (r_) return r_;     \
    } while (0)

// ---- validation of one scenario ------------------------------------------
int validate(MossHandle* h, const MossNetwork* net, const MossVehicles* veh, const MossParams* p,
             std::vector<std::vector<int32_t>>* road_out) {
    if (!net || !veh || !p) return fail(h, MOSS_EINVAL, "null argument");
    if (p->delta != 4.0) return fail(h, MOSS_EINVAL, "only delta = 4 is supported");
    if (p->precision != 32 && p->precision != 64) return fail(h, MOSS_EINVAL, "precision must be 32 or 64");
    if (!(p->dt > 0) || !(p->a_max > 0) || !(p->b_comf > 0) || !(p->s0 >= 0) || !(p->veh_len > 0) ||
        !(p->T >= 0))
        return fail(h, MOSS_EINVAL, "invalid model parameter");
    const int R = net->n_roads, NRL = net->n_road_lanes, NL = net->n_lanes, J = net->n_junctions;
    if (R < 1 || NRL < 1 || NL < NRL || J < 0) return fail(h, MOSS_EINVAL, "bad network sizes");
    if (!net->road_lane_off || !net->lane_length || !net->lane_vmax || !net->jl_off)
        return fail(h, MOSS_EINVAL, "missing network array");
    if (NL > NRL && (!net->jl_target || !net->jl_junction || !net->jl_mask))
        return fail(h, MOSS_EINVAL, "missing junction-lane array");
    if (J > 0 && (!net->junc_offset || !net->junc_phase_off))
        return fail(h, MOSS_EINVAL, "missing junction array");
    if (net->road_lane_off[0] != 0 || net->road_lane_off[R] != NRL)
        return fail(h, MOSS_EINVAL, "road_lane_off must start at 0 and end at n_road_lanes");
    for (int r = 0; r < R; ++r)
        if (net->road_lane_off[r + 1] <= net->road_lane_off[r])
            return fail(h, MOSS_EINVAL, "every road needs at least one lane");
    for (int l = 0; l < NL; ++l)
        if (!(net->lane_length[l] > 0.f) || !(net->lane_vmax[l] > 0.f) || !std::isfinite(net->lane_length[l]))
            return fail(h, MOSS_EINVAL, "lane lengths and speed limits must be > 0");
    if (net->jl_off[0] != NRL || net->jl_off[NRL] != NL) return fail(h, MOSS_EINVAL, "jl_off range");
    for (int l = 0; l < NRL; ++l)
        if (net->jl_off[l + 1] < net->jl_off[l]) return fail(h, MOSS_EINVAL, "jl_off not monotone");
    int nph = 0;
    if (J > 0) {
        if (net->junc_phase_off[0] != 0) return fail(h, MOSS_EINVAL, "junc_phase_off[0] != 0");
        for (int j = 0; j < J; ++j) {
            const int np = net->junc_phase_off[j + 1] - net->junc_phase_off[j];
            if (np < 0 || np > 8) return fail(h, MOSS_EINVAL, "a junction has 0..8 phases");
        }
        nph = net->junc_phase_off[J];
        if (nph > 0 && (!net->phase_green || !net->phase_amber)) return fail(h, MOSS_EINVAL, "missing phases");
        for (int k = 0; k < nph; ++k)
            if (net->phase_green[k] < 0 || net->phase_amber[k] < 0)
                return fail(h, MOSS_EINVAL, "negative phase duration");
    }
    std::vector<int32_t> road_of(NRL);
    for (int r = 0; r < R; ++r)
        for (int l = net->road_lane_off[r]; l < net->road_lane_off[r + 1]; ++l) road_of[l] = r;
    for (int j = NRL; j < NL; ++j) {
        const int k = j - NRL;
        if (net->jl_target[k] < 0 || net->jl_target[k] >= NRL) return fail(h, MOSS_EINVAL, "jl_target range");
        if (net->jl_junction[k] < 0 || net->jl_junction[k] >= J) return fail(h, MOSS_EINVAL, "jl_junction range");
        if (net->jl_mask[k] < 0 || net->jl_mask[k] > 255) return fail(h, MOSS_EINVAL, "jl_mask must fit 8 bits");
        if (net->jl_plans && (net->jl_plans[k] < 0 || net->jl_plans[k] > 255))
            return fail(h, MOSS_EINVAL, "jl_plans must fit 8 bits");
    }
    // out-roads reachable from some lane of each road (a vehicle on a lane
    // without access changes lanes towards the group that has it, R27)
    road_out->assign(R, {});
    for (int r = 0; r < R; ++r) {
        std::vector<int32_t> common;
        for (int l = net->road_lane_off[r]; l < net->road_lane_off[r + 1]; ++l) {
            std::vector<int32_t> outs;
            for (int j = net->jl_off[l]; j < net->jl_off[l + 1]; ++j)
                outs.push_back(road_of[net->jl_target[j - NRL]]);
            std::sort(outs.begin(), outs.end());
            if (std::adjacent_find(outs.begin(), outs.end()) != outs.end())
                return fail(h, MOSS_EINVAL, "a lane has two junction lanes to the same road");
            std::vector<int32_t> x;
            std::set_union(common.begin(), common.end(), outs.begin(), outs.end(), std::back_inserter(x));
            common.swap(x);
        }
        (*road_out)[r] = common;
    }
    const int N = veh->n;
    if (N < 0 || N >= (1 << 30)) return fail(h, MOSS_EINVAL, "vehicle count out of range");
    if (N > 0 && (!veh->route_off || !veh->routes || !veh->start_lane || !veh->dep || !veh->v0f))
        return fail(h, MOSS_EINVAL, "missing vehicle array");
    if (N > 0 && veh->route_off[0] != 0) return fail(h, MOSS_EINVAL, "route_off[0] != 0");
    for (int i = 0; i < N; ++i) {
        const int a = veh->route_off[i], b = veh->route_off[i + 1];
        if (b <= a) return fail(h, MOSS_EINVAL, "every route needs at least one road");
        for (int k = a; k < b; ++k)
            if (veh->routes[k] < 0 || veh->routes[k] >= R) return fail(h, MOSS_EINVAL, "route road out of range");
        for (int k = a; k + 1 < b; ++k) {
            const auto& o = (*road_out)[veh->routes[k]];
            if (!std::binary_search(o.begin(), o.end(), veh->routes[k + 1]))
                return fail(h, MOSS_EINVAL, "route of vehicle " + std::to_string(i) +
                                                " uses a turn no lane of the road has");
        }
        const int sl = veh->start_lane[i];
        if (sl < 0 || sl >= NRL || road_of[sl] != veh->routes[a])
            return fail(h, MOSS_EINVAL, "start lane must be a lane of the first road");
        if (veh->dep[i] < 0) return fail(h, MOSS_EINVAL, "negative departure step");
        if (!(veh->v0f[i] > 0.f) || !std::isfinite(veh->v0f[i])) return fail(h, MOSS_EINVAL, "v0f must be > 0");
    }
    return MOSS_OK;
}

bool same_model(const MossParams& a, const MossParams& b) {
    return a.dt == b.dt && a.a_max == b.a_max && a.b_comf == b.b_comf && a.T == b.T && a.s0 == b.s0 &&
           a.delta == b.delta && a.veh_len == b.veh_len && a.politeness == b.politeness &&
           a.a_th == b.a_th && a.b_safe == b.b_safe && a.p_attempt == b.p_attempt && a.p_hi == b.p_hi &&
           a.p_lo == b.p_lo && a.flag_band == b.flag_band && a.precision == b.precision;
}

size_t reca_size(int precision) { return precision == 64 ? sizeof(RecA<double>) : sizeof(RecA<float>); }
size_t sv_size(int precision) { return precision == 64 ? sizeof(SV<double>) : sizeof(SV<float>); }

template <typename Real>
Ctx<Real> make_ctx(MossHandle* h, int cur) {
    Ctx<Real> c;
    std::memset(&c, 0, sizeof(c));
    c.n_lanes = h->n_lanes; c.n_junctions = h->n_junctions; c.n_scen = h->n_scen; c.n_veh = h->n_veh;
    c.lane = h->d_lane;
    c.junc = h->d_junc;
    c.phase_green = h->d_phase_green; c.phase_amber = h->d_phase_amber;
    c.junc_policy = h->d_junc_policy; c.junc_manual = h->d_junc_manual; c.junc_state = h->d_junc_state;
    c.mp = h->d_mp; c.jj_off = h->d_jj_off; c.jj_lane = h->d_jj_lane; c.jj_from = h->d_jj_from;
    c.n_jj = h->n_jj; c.mp_press = h->d_mp_press; c.n_mp = &h->d_cnt[0].n_mp;
    c.road_span = h->d_road_span;
    c.route_span = h->d_route_span; c.routes = h->d_routes; c.dep = h->d_dep; c.v0f = h->d_v0f;
    c.vstatus = h->d_vstatus; c.vflags = h->d_vflags;
    c.q_off = h->d_q_off; c.q_ids = h->d_q_ids; c.q_head = h->d_q_head;
    c.start_lanes = h->d_start_lanes; c.n_start = (int)h->start_lanes.size();
    c.key0 = h->d_key0; c.key1 = h->d_key1; c.veh_base = h->d_veh_base; c.scen_step = h->d_step;
    c.metrics = h->d_metrics;
    for (int k = 0; k < 2; ++k) {
        const SnapBufs& b = h->snap[k == 0 ? cur : 1 - cur];
        Snap<Real>& s = k == 0 ? c.cur : c.nxt;
        s.a = (RecA<Real>*)b.a; s.b = b.b; s.off = b.off;
    }
    c.code = h->d_code; c.stay = (SV<Real>*)h->d_stay;
    c.ea = (RecA<Real>*)h->d_ea; c.eb = h->d_eb; c.enext = h->d_enext; c.head = h->d_head;
    c.enter = h->d_enter; c.leave = h->d_leave; c.lbefore = h->d_lbefore;
    c.tile_leave = h->d_tile_leave; c.tile_prefix = h->d_tile_prefix; c.lane_tiles = h->d_lane_tiles;
    c.cands = (Cand<Real>*)h->d_cands; c.gap_head = h->d_gap_head;
    c.n_lane_tiles = h->n_lane_tiles; c.max_slot_tiles = h->max_slot_tiles;
    c.n_junc_chunks = h->n_junc_chunks; c.cnt = h->d_cnt + cur;
    c.cnt_next = h->d_cnt + (1 - cur); c.err = &h->d_cnt[0].err;
    const MossParams& p = h->prm;
    c.dt = Real(p.dt); c.a_max = Real(p.a_max); c.b_comf = Real(p.b_comf); c.T = Real(p.T);
    c.s0 = Real(p.s0); c.len = Real(p.veh_len); c.pol = Real(p.politeness); c.a_th = Real(p.a_th);
    c.b_safe = Real(p.b_safe); c.p_att = Real(p.p_attempt); c.p_hi = Real(p.p_hi); c.p_lo = Real(p.p_lo);
    c.band = Real(p.flag_band);
    c.inv_2sqrt_ab = Real(1.0 / (2.0 * std::sqrt(p.a_max * p.b_comf)));
    return c;
}

struct Grids {
    int decide_work, decide_ins, resolve, lanescan, place;
};

Grids grids(const MossHandle* h) {
    Grids g;
    g.decide_work = std::max(1, std::min(h->max_slot_tiles, h->sm_count * h->cfg_decide));
    const int ns = (int)h->start_lanes.size();
    g.decide_ins = ns > 0 ? (ns + TILE - 1) / TILE : 0;  // one start lane per thread
    // candidates are a few per cent of the vehicles; the kernel strides over them
    g.resolve = std::max(1, std::min(h->max_slot_tiles, h->sm_count * 2));
    const int tickets = h->n_lane_tiles + 1 + h->n_junc_chunks;
    g.lanescan = std::max(1, std::min(tickets, h->sm_count * h->cfg_lanescan));
    g.place = std::max(1, std::min(2 * h->max_slot_tiles, h->sm_count * h->cfg_place));
    return g;
}

template <typename Real>
void enqueue_step(MossHandle* h, int cur, bool timed) {
    Ctx<Real> c = make_ctx<Real>(h, cur);
    const Grids g = grids(h);
    cudaStream_t s = h->stream;
    if (timed) cudaEventRecord(h->ev[0], s);
    if (h->lane_groups) k_decide<Real, true><<<g.decide_work + g.decide_ins, TILE, 0, s>>>(c, g.decide_work);
    else k_decide<Real, false><<<g.decide_work + g.decide_ins, TILE, 0, s>>>(c, g.decide_work);
    if (timed) cudaEventRecord(h->ev[1], s);
#if !MOSS_FOLD_RESOLVE
    k_resolve<Real><<<g.resolve, TILE, 0, s>>>(c);
#endif
    if (timed) cudaEventRecord(h->ev[2], s);
    k_lanescan<Real><<<g.lanescan, LANESCAN_THREADS, 0, s>>>(c);
    if (timed) cudaEventRecord(h->ev[3], s);
    k_place<Real><<<g.place, TILE, 0, s>>>(c);
    if (timed) cudaEventRecord(h->ev[4], s);
}

void enqueue(MossHandle* h, int cur, bool timed) {
    if (h->precision == 64) enqueue_step<double>(h, cur, timed);
    else enqueue_step<float>(h, cur, timed);
}

template <typename Real>
void enqueue_junction_init(MossHandle* h) {
    Ctx<Real> c = make_ctx<Real>(h, h->parity);
    const int nb = std::max(1, std::min((h->n_junctions + 255) / 256, h->sm_count * 4));
    k_junction_init<Real><<<nb, 256, 0, h->stream>>>(c);
}

int junction_init(MossHandle* h) {
    if (h->n_junctions == 0) return MOSS_OK;
    if (h->precision == 64) enqueue_junction_init<double>(h);
    else enqueue_junction_init<float>(h);
    CK(cudaGetLastError());
    return MOSS_OK;
}

template <typename Real>
void enqueue_set_signal(MossHandle* h, int n, int policy) {
    Ctx<Real> c = make_ctx<Real>(h, h->parity);
    k_set_signal<Real><<<(n + 255) / 256, 256, 0, h->stream>>>(c, n, h->d_stage, h->d_stage + n, policy);
}

void destroy_graphs(MossHandle* h) {
    for (int k = 0; k < 2; ++k) {
        if (h->g2[k]) cudaGraphExecDestroy(h->g2[k]);
        if (h->g1[k]) cudaGraphExecDestroy(h->g1[k]);
        h->g2[k] = h->g1[k] = nullptr;
    }
}

int build_graphs(MossHandle* h) {
    for (int p = 0; p < 2; ++p) {
        for (int nsteps = 1; nsteps <= 2; ++nsteps) {
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            for (int k = 0; k < nsteps; ++k) enqueue(h, (p + k) & 1, false);
            CK(cudaStreamEndCapture(h->stream, &g));
            cudaGraphExec_t ex = nullptr;
            cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
            (nsteps == 2 ? h->g2[p] : h->g1[p]) = ex;
        }
    }
    return MOSS_OK;
}

// read back the device error word; recoverable reports are cleared once read,
// a poisoning error stays (every later step of the handle is skipped)
// the device error word, already read back: a status (a recoverable error is
// cleared on the device; the poison bit stays)
int device_status(MossHandle* h, int err) {
    if (err == 0) return MOSS_OK;
    if (!(err & ERR_POISON)) {
        const int zero = 0;
        CK(cudaMemcpy(&h->d_cnt->err, &zero, sizeof(int), cudaMemcpyHostToDevice));
    }
    if (err & ERR_TIMEOUT) return fail(h, MOSS_ETIMEOUT, "a bounded device wait gave up");
    std::string m = "device reported:";
    if (err & ERR_ROUTE) m += " undrivable route;";
    if (err & ERR_TRANSFER) m += " transfer overflow;";
    if (err & ERR_RANGE) m += " index out of range;";
    return fail(h, MOSS_EDEVICE, m);
}

int check_device(MossHandle* h) {
    int err = 0;
    CK(cudaMemcpy(&err, &h->d_cnt->err, sizeof(int), cudaMemcpyDeviceToHost));
    return device_status(h, err);
}

// ---- create (n scenarios as one union network) ------------------------------
int create_impl(int n, const MossNetwork* nets, const MossVehicles* vehs, const MossParams* prms,
                void* stream, MossHandle* h) {
    if (n < 1) return fail(h, MOSS_EINVAL, "need at least one scenario");
    if (n > 65535) return fail(h, MOSS_EINVAL, "at most 65535 scenarios in a batch");
    h->prm = prms[0];
    h->precision = prms[0].precision;
    h->n_scen = n;
    for (int k = 1; k < n; ++k)
        if (!same_model(prms[0], prms[k]))
            return fail(h, MOSS_EINVAL, "batched scenarios must share the model parameters");
    long long tot_lanes = 0, tot_j = 0, tot_v = 0, tot_routes = 0, tot_ph = 0, tot_roads = 0;
    std::vector<std::vector<std::vector<int32_t>>> outs(n);
    for (int k = 0; k < n; ++k) {
        TRY(validate(h, &nets[k], &vehs[k], &prms[k], &outs[k]));
        tot_lanes += nets[k].n_lanes; tot_j += nets[k].n_junctions; tot_v += vehs[k].n;
        tot_routes += vehs[k].n ? vehs[k].route_off[vehs[k].n] : 0;
        tot_ph += nets[k].n_junctions ? nets[k].junc_phase_off[nets[k].n_junctions] : 0;
        tot_roads += nets[k].n_roads;
    }
    if (tot_lanes >= (1ll << 30) || tot_v >= (1ll << 30) || tot_routes >= (1ll << 31) - 1 ||
        tot_roads >= (1ll << 30))
        return fail(h, MOSS_EINVAL, "batch too large for 32-bit indices");
    h->n_lanes = (int)tot_lanes; h->n_junctions = (int)tot_j; h->n_veh = (int)tot_v;
    h->n_phases = (int)tot_ph;
    const int NL = h->n_lanes, NJ = h->n_junctions, NV = h->n_veh;
    h->lanes.resize(NL);
    h->lane_src_road.assign(NL, -1);
    h->junc_scen.resize(NJ); h->junc_phase_off.resize(NJ + 1);
    std::vector<int32_t> junc_offset(NJ), phase_green(tot_ph), phase_amber(tot_ph);
    h->route_span.resize(NV); h->routes.resize(tot_routes); h->dep.resize(NV);
    h->start_lane.resize(NV); h->v0f.resize(NV); h->veh_scen.resize(NV);
    h->scen_veh_off.assign(n + 1, 0); h->scen_lane_off.assign(n + 1, 0); h->scen_junc_off.assign(n + 1, 0);
    h->scen_road_off.assign(n + 1, 0);
    h->jl_plans.assign(tot_lanes, 0xff);
    h->road_span.assign(tot_roads, make_int2(0, 0));
    h->key0.resize(n); h->key1.resize(n);
    int LO = 0, JO = 0, VO = 0, RO = 0, PO = 0, ROFF = 0;
    for (int k = 0; k < n; ++k) {
        const MossNetwork& nt = nets[k];
        const MossVehicles& vh = vehs[k];
        const int NRL = nt.n_road_lanes;
        std::vector<int32_t> road_of(NRL);
        for (int r = 0; r < nt.n_roads; ++r)
            for (int l = nt.road_lane_off[r]; l < nt.road_lane_off[r + 1]; ++l) road_of[l] = r;
        for (int l = 0; l < nt.n_lanes; ++l) {
            LaneInfo& li = h->lanes[LO + l];
            li.scen = k;
            li.L = nt.lane_length[l];
            li.vmax = nt.lane_vmax[l];
            if (l < NRL) {
                const int r = road_of[l];
                li.lo = LO + nt.road_lane_off[r];
                li.hi = LO + nt.road_lane_off[r + 1];
                li.jb = LO + nt.jl_off[l];
                li.je = LO + nt.jl_off[l + 1];
                li.road = RO + r;
            } else {
                const int q = l - NRL;
                li.lo = -1;
                li.hi = LO + nt.jl_target[q];
                li.jb = JO + nt.jl_junction[q];
                li.je = nt.jl_mask[q];
                li.road = RO + road_of[nt.jl_target[q]];
            }
        }
        for (int l = 0; l < NRL; ++l)
            for (int j = nt.jl_off[l]; j < nt.jl_off[l + 1]; ++j) h->lane_src_road[LO + j] = RO + road_of[l];
        for (int r = 0; r < nt.n_roads; ++r)
            h->road_span[RO + r] = make_int2(LO + nt.road_lane_off[r], LO + nt.road_lane_off[r + 1]);
        if (nt.jl_plans) {
            h->lane_groups = true;  // a plan can take a turn away from some lanes
            for (int q = 0; q < nt.n_lanes - NRL; ++q) {
                h->jl_plans[LO + NRL + q] = nt.jl_plans[q];
                if (!(nt.jl_plans[q] & 1)) h->lanes[LO + NRL + q].flags |= LF_OFF;  // roads start in plan 0
            }
        }
        for (int j = 0; j < nt.n_junctions; ++j) {
            h->junc_scen[JO + j] = k;
            junc_offset[JO + j] = nt.junc_offset[j];
            h->junc_phase_off[JO + j] = PO + nt.junc_phase_off[j];
        }
        const int nph = nt.n_junctions ? nt.junc_phase_off[nt.n_junctions] : 0;
        for (int q = 0; q < nph; ++q) {
            phase_green[PO + q] = nt.phase_green[q];
            phase_amber[PO + q] = nt.phase_amber[q];
        }
        for (int i = 0; i < vh.n; ++i) {
            const int g = VO + i;
            const int a = vh.route_off[i], b = vh.route_off[i + 1];
            for (int q = a; q < b; ++q) h->routes[ROFF + q] = RO + vh.routes[q];
            h->route_span[g] = make_int2(ROFF + a, ROFF + b);
            h->dep[g] = vh.dep[i];
            h->start_lane[g] = LO + vh.start_lane[i];
            h->v0f[g] = vh.v0f[i];
            h->veh_scen[g] = k;
        }
        h->key0[k] = (uint32_t)(prms[k].seed & 0xffffffffull);
        h->key1[k] = (uint32_t)(prms[k].seed >> 32) ^ prms[k].scenario;
        ROFF += vh.n ? vh.route_off[vh.n] : 0;
        LO += nt.n_lanes; JO += nt.n_junctions; VO += vh.n; RO += nt.n_roads; PO += nph;
        h->scen_veh_off[k + 1] = VO; h->scen_lane_off[k + 1] = LO; h->scen_junc_off[k + 1] = JO;
        h->scen_road_off[k + 1] = RO;
    }
    h->junc_phase_off[NJ] = PO;
    // departure queues per start lane ordered by (dep, id) (R18)
    h->q_off.assign(NL + 1, 0);
    for (int i = 0; i < NV; ++i) h->q_off[h->start_lane[i] + 1]++;
    for (int l = 0; l < NL; ++l) h->q_off[l + 1] += h->q_off[l];
    h->q_ids.resize(NV);
    {
        std::vector<int32_t> fill(h->q_off.begin(), h->q_off.end() - 1);
        for (int i = 0; i < NV; ++i) h->q_ids[fill[h->start_lane[i]]++] = i;
        for (int l = 0; l < NL; ++l)
            std::stable_sort(h->q_ids.begin() + h->q_off[l], h->q_ids.begin() + h->q_off[l + 1],
                             [&](int a, int b) { return h->dep[a] < h->dep[b]; });
    }
    h->start_lanes.clear();
    for (int l = 0; l < NL; ++l)
        if (h->q_off[l + 1] > h->q_off[l]) h->start_lanes.push_back(l);

    // lane groups: a road with a turn not served by all of its lanes
    for (size_t r = 0; r < h->road_span.size() && !h->lane_groups; ++r) {
        const int2 sp = h->road_span[r];
        std::vector<int> all, first;
        for (int l = sp.x; l < sp.y; ++l) {
            std::vector<int> outs;
            for (int j = h->lanes[l].jb; j < h->lanes[l].je; ++j) outs.push_back(h->lanes[j].road);
            std::sort(outs.begin(), outs.end());
            if (l == sp.x) first = outs;
            else if (outs != first) h->lane_groups = true;
        }
    }

    // ---- device
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    CK(cudaGetDevice(&h->device));
    CK(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));
    TRY(upload(h, &h->d_lane, h->lanes));
    std::vector<JuncInfo> junc(NJ);
    for (int j = 0; j < NJ; ++j) {
        junc[j].offset = junc_offset[j];
        junc[j].phase_off = h->junc_phase_off[j];
        junc[j].np = h->junc_phase_off[j + 1] - h->junc_phase_off[j];
        junc[j].scen = h->junc_scen[j];
    }
    TRY(upload(h, &h->d_junc, junc));
    TRY(upload(h, &h->d_phase_green, phase_green));
    TRY(upload(h, &h->d_phase_amber, phase_amber));
    TRY(upload(h, &h->d_junc_policy, std::vector<int32_t>(NJ, POL_FIXED)));
    TRY(upload(h, &h->d_junc_manual, std::vector<int32_t>(NJ, 0)));
    TRY(dalloc(h, &h->d_junc_state, NJ));
    {
        // junction lanes of every junction with the road lane each one leaves
        // (the pressures of the max-pressure policy)
        std::vector<int32_t> from(NL, -1), jj_off(NJ + 1, 0);
        for (int l = 0; l < NL; ++l)
            if (h->lanes[l].lo >= 0)
                for (int q = h->lanes[l].jb; q < h->lanes[l].je; ++q) from[q] = l;
        for (int l = 0; l < NL; ++l)
            if (h->lanes[l].lo < 0) jj_off[h->lanes[l].jb + 1]++;
        for (int j = 0; j < NJ; ++j) jj_off[j + 1] += jj_off[j];
        std::vector<int32_t> jj_lane(std::max(jj_off[NJ], 1)), jj_from(std::max(jj_off[NJ], 1));
        std::vector<int32_t> fill(jj_off.begin(), jj_off.end() - 1);
        for (int l = 0; l < NL; ++l)
            if (h->lanes[l].lo < 0) {
                const int q = fill[h->lanes[l].jb]++;
                jj_lane[q] = l;
                jj_from[q] = from[l];
            }
        TRY(upload(h, &h->d_jj_off, jj_off));
        TRY(upload(h, &h->d_jj_lane, jj_lane));
        TRY(upload(h, &h->d_jj_from, jj_from));
        TRY(upload(h, &h->d_mp, std::vector<int4>(std::max(NJ, 1), make_int4(0, 1, -1, 0))));
        TRY(upload(h, &h->d_mp_press, std::vector<int32_t>((size_t)std::max(NJ, 1) * 8, 0)));
        std::vector<int2> span(h->road_span);
        if (span.empty()) span.push_back(make_int2(0, 0));
        TRY(upload(h, &h->d_road_span, span));
        TRY(dalloc(h, &h->d_lstage, 2 * (size_t)std::max(NL, 1)));
        TRY(upload(h, &h->d_jl_plans, h->jl_plans.empty() ? std::vector<int32_t>(1, 0xff) : h->jl_plans));
        TRY(upload(h, &h->d_road_mark, std::vector<int8_t>(std::max<long long>(tot_roads, 1), 0)));
        TRY(dalloc(h, (char**)&h->d_mbuf, sizeof(double) * (size_t)std::max(std::max(NL, (int)tot_roads), 1)));
        h->n_jj = jj_off[NJ];
    }
    {
        std::vector<int2> span(h->route_span);
        if (span.empty()) span.push_back(make_int2(0, 0));
        TRY(upload(h, &h->d_route_span, span));
        // room for re-routed vehicles' routes (grown on demand)
        h->routes_cap = h->routes.size() + std::max<size_t>(h->routes.size() / 4, 1 << 16);
        TRY(dalloc(h, &h->d_routes, h->routes_cap));
        if (!h->routes.empty())
            CK(cudaMemcpy(h->d_routes, h->routes.data(), h->routes.size() * 4, cudaMemcpyHostToDevice));
    }
    TRY(upload(h, &h->d_dep, h->dep));
    TRY(upload(h, &h->d_v0f, h->v0f));
    TRY(upload(h, &h->d_vstatus, std::vector<int32_t>(NV, MOSS_ST_WAITING)));
    TRY(upload(h, &h->d_req, std::vector<int32_t>(std::max(NV, 1), -1)));
    TRY(upload(h, &h->d_vflags, std::vector<int32_t>(NV, 0)));
    TRY(upload(h, &h->d_q_off, h->q_off));
    TRY(upload(h, &h->d_q_ids, h->q_ids));
    TRY(upload(h, &h->d_q_head, std::vector<int32_t>(h->q_off.begin(), h->q_off.end() - 1)));
    TRY(upload(h, &h->d_start_lanes, h->start_lanes));
    TRY(upload(h, &h->d_key0, h->key0));
    TRY(upload(h, &h->d_key1, h->key1));
    TRY(upload(h, &h->d_veh_base, std::vector<int32_t>(h->scen_veh_off.begin(), h->scen_veh_off.end() - 1)));
    TRY(upload(h, &h->d_step, std::vector<long long>(n, 0)));
    TRY(upload(h, &h->d_metrics, std::vector<long long>((size_t)n * M_NFIELDS, 0)));
    const size_t cap = std::max(NV, 1);
    const size_t ra = reca_size(h->precision);
    for (int k = 0; k < 2; ++k) {
        SnapBufs& b = h->snap[k];
        TRY(dalloc(h, (char**)&b.a, cap * ra));
        TRY(dalloc(h, &b.b, cap));
        TRY(upload(h, &b.off, std::vector<int32_t>(NL + 1, 0)));
    }
    TRY(dalloc(h, &h->d_code, cap));
    TRY(dalloc(h, (char**)&h->d_stay, cap * sv_size(h->precision)));
    TRY(dalloc(h, (char**)&h->d_ea, cap * ra));
    TRY(dalloc(h, &h->d_eb, cap));
    TRY(dalloc(h, &h->d_enext, cap));
    TRY(dalloc(h, (char**)&h->d_cands,
               cap * (h->precision == 64 ? sizeof(Cand<double>) : sizeof(Cand<float>))));
    TRY(upload(h, &h->d_gap_head, std::vector<unsigned long long>(cap + NL + 1, 0ull)));
    TRY(upload(h, &h->d_head, std::vector<unsigned long long>(NL, 0ull)));
    TRY(upload(h, &h->d_enter, std::vector<int32_t>(NL, 0)));
    TRY(upload(h, &h->d_leave, std::vector<int32_t>(NL, 0)));
    TRY(dalloc(h, &h->d_lbefore, NL));
    h->n_lane_tiles = (NL + LANESCAN_TILE - 1) / LANESCAN_TILE;
    h->max_slot_tiles = (NV + TILE - 1) / TILE + 1;
    // tile counter arrays padded for the 16-byte loads of the tile-prefix scan
    const int tile_cap = ((h->max_slot_tiles + 4 * LANESCAN_THREADS - 1) / (4 * LANESCAN_THREADS)) *
                         (4 * LANESCAN_THREADS);
    h->n_junc_chunks = (NJ + JUNC_CHUNK - 1) / JUNC_CHUNK;
    TRY(upload(h, &h->d_tile_leave, std::vector<int32_t>(tile_cap, 0)));
    TRY(upload(h, &h->d_tile_prefix, std::vector<int32_t>(tile_cap, 0)));
    TRY(upload(h, &h->d_lane_tiles, std::vector<unsigned long long>(h->n_lane_tiles, 0ull)));
    std::vector<Counters> c0(2, Counters{});
    c0[0].tag = 1;
    TRY(upload(h, &h->d_cnt, c0));
    TRY(dalloc(h, &h->d_stage, 2 * std::max(NJ, 1)));
    CK(cudaHostAlloc((void**)&h->h_stage, sizeof(int32_t) * 2 * std::max(NJ, 1), cudaHostAllocDefault));
    CK(cudaHostAlloc((void**)&h->h_rb, sizeof(long long) * RB_WORDS * (MOSS_METRIC_SLOTS + 1),
                     cudaHostAllocDefault));
    for (int k = 0; k < MOSS_METRIC_SLOTS; ++k)
        CK(cudaEventCreateWithFlags(&h->rb_ev[k], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->stage_free, cudaEventDisableTiming));
    CK(cudaEventRecord(h->stage_free, h->stream));
    for (int k = 0; k <= N_STEP_KERNELS; ++k) CK(cudaEventCreate(&h->ev[k]));
    TRY(junction_init(h));
    CK(cudaStreamSynchronize(h->stream));
    TRY(build_graphs(h));
    return MOSS_OK;
}

void free_all(MossHandle* h) {
    destroy_graphs(h);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& a : h->allocs) raw_free(h, a.first, a.second);
    h->allocs.clear();
    for (int k = 0; k <= N_STEP_KERNELS; ++k)
        if (h->ev[k]) cudaEventDestroy(h->ev[k]);
    if (h->stage_free) cudaEventDestroy(h->stage_free);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    h->h_stage = nullptr;
    if (h->h_rb) cudaFreeHost(h->h_rb);
    h->h_rb = nullptr;
    for (int k = 0; k < MOSS_METRIC_SLOTS; ++k)
        if (h->rb_ev[k]) cudaEventDestroy(h->rb_ev[k]);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->stream = nullptr;
}

// copies of scenario s's metric record, its step and the device error word,
// behind the work queued so far, into readback slot `slot`
int enqueue_readback(MossHandle* h, int s, int slot) {
    long long* M = h->h_rb + (size_t)slot * RB_WORDS;
    CK(cudaMemcpyAsync(M, h->d_metrics + (size_t)s * M_NFIELDS, M_NFIELDS * sizeof(long long),
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(M + M_NFIELDS, h->d_step + s, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(M + M_NFIELDS + 1, &h->d_cnt->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    return MOSS_OK;
}

// the metrics of scenario s from a completed readback slot
int readback_metrics(MossHandle* h, int s, int slot, MossMetrics* out) {
    const long long* M = h->h_rb + (size_t)slot * RB_WORDS;
    const long long step = M[M_NFIELDS];
    int err = 0;
    std::memcpy(&err, M + M_NFIELDS + 1, sizeof(int));
    const int nv = h->scen_veh_off[s + 1] - h->scen_veh_off[s];
    out->step = step;
    out->n_active = M[M_CUR_ACTIVE];
    out->n_waiting = nv - M[M_CUR_ACTIVE] - M[M_CUR_ARRIVED];
    out->n_arrived = M[M_ARRIVED];
    out->tt_sum = (double)M[M_TT_STEPS] * h->prm.dt;
    out->speed_sum = (double)M[M_SPEED_FX] / SPEED_FX;
    out->vehicle_updates = M[M_UPDATES];
    out->lane_changes = M[M_LANE_CHANGES];
    out->flagged = M[M_FLAGGED];
    out->overlaps = M[M_OVERLAPS];
    out->inserted = M[M_INSERTED];
    out->errors = M[M_ERRORS];
    out->mobil_evals = M[M_MOBIL];
    return device_status(h, err);
}

int scen_metrics(MossHandle* h, int s, MossMetrics* out) {
    if (!out) return fail(h, MOSS_EINVAL, "null output");
    if (s < 0 || s >= h->n_scen) return fail(h, MOSS_EINVAL, "scenario index out of range");
    // one stream round trip: the copies go behind the queued work, one wait
    TRY(enqueue_readback(h, s, MOSS_METRIC_SLOTS));
    CK(cudaStreamSynchronize(h->stream));
    return readback_metrics(h, s, MOSS_METRIC_SLOTS, out);
}

template <typename Real>
void unpack_a(const std::vector<char>& raw, int n, std::vector<int32_t>& lane, std::vector<int32_t>& id,
              std::vector<double>& sv, std::vector<double>& vv) {
    const RecA<Real>* a = (const RecA<Real>*)raw.data();
    for (int k = 0; k < n; ++k) {
        lane[k] = a[k].lane; id[k] = a[k].id; sv[k] = (double)a[k].s; vv[k] = (double)a[k].v;
    }
}

int scen_state(MossHandle* h, int s, MossState* out) {
    if (!out || !out->status || !out->lane || !out->s || !out->v || !out->rc || !out->flags)
        return fail(h, MOSS_EINVAL, "null state array");
    if (s < 0 || s >= h->n_scen) return fail(h, MOSS_EINVAL, "scenario index out of range");
    CK(cudaStreamSynchronize(h->stream));
    Counters c;
    CK(cudaMemcpy(&c, h->d_cnt + h->parity, sizeof(c), cudaMemcpyDeviceToHost));
    const int n = c.n_cur, NV = h->n_veh;
    const SnapBufs& b = h->snap[h->parity];
    const size_t ra = reca_size(h->precision);
    std::vector<char> raw((size_t)n * ra);
    std::vector<RecB> rb(n);
    std::vector<int32_t> lane(n), id(n), status(NV), vflags(NV);
    std::vector<double> sv(n), vv(n);
    long long step = 0;
    CK(cudaMemcpy(&step, h->d_step + s, sizeof(long long), cudaMemcpyDeviceToHost));
    if (n > 0) {
        CK(cudaMemcpy(raw.data(), b.a, raw.size(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(rb.data(), b.b, n * sizeof(RecB), cudaMemcpyDeviceToHost));
        if (h->precision == 64) unpack_a<double>(raw, n, lane, id, sv, vv);
        else unpack_a<float>(raw, n, lane, id, sv, vv);
    }
    CK(cudaMemcpy(status.data(), h->d_vstatus, NV * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(vflags.data(), h->d_vflags, NV * 4, cudaMemcpyDeviceToHost));
    const int v0 = h->scen_veh_off[s], v1 = h->scen_veh_off[s + 1];
    const int lo = h->scen_lane_off[s];
    const long long tag = (step - 1) & 0xFFFFFF;
    for (int g = v0; g < v1; ++g) {
        const int i = g - v0;
        out->status[i] = status[g];
        out->lane[i] = -1; out->s[i] = 0; out->v[i] = 0; out->rc[i] = 0;
        out->flags[i] = ((long long)(((unsigned)vflags[g]) >> 8) == tag && step > 0) ? (vflags[g] & 255) : 0;
    }
    for (int k = 0; k < n; ++k) {
        const int g = id[k];
        if (g < v0 || g >= v1) continue;
        const int i = g - v0;
        out->lane[i] = lane[k] - lo;
        out->s[i] = sv[k];
        out->v[i] = vv[k];
        out->rc[i] = rb[k].rptr - h->route_span[g].x;
    }
    return check_device(h);
}

int jl_toward_host(const MossHandle* h, int l, int out_road) {
    for (int j = h->lanes[l].jb; j < h->lanes[l].je; ++j)
        if (h->lanes[j].road == out_road && !(h->lanes[j].flags & LF_OFF)) return j;
    return -1;
}

template <typename Real>
int upload_state(MossHandle* h, const std::vector<int>& order, const std::vector<double>& s,
                 const std::vector<double>& v, const std::vector<int>& lane_of, const std::vector<int>& rc) {
    const int n = (int)order.size();
    std::vector<RecA<Real>> a(n);
    std::vector<RecB> b(n);
    std::vector<int32_t> off(h->n_lanes + 1, 0);
    for (int k = 0; k < n; ++k) {
        const int g = order[k];
        const int l = lane_of[g];
        std::memset(&a[k], 0, sizeof(a[k]));
        a[k].s = Real(s[g]); a[k].v = Real(v[g]); a[k].id = g; a[k].lane = l;
        b[k].v0f = h->v0f[g];
        b[k].rptr = h->route_span[g].x + rc[g];
        b[k].rlast = h->route_span[g].y - 1;
        if (h->lanes[l].lo < 0) b[k].nl = h->lanes[l].hi;
        else b[k].nl = b[k].rptr < b[k].rlast ? jl_toward_host(h, l, h->routes[b[k].rptr + 1]) : -1;
        off[l + 1]++;
    }
    for (int l = 0; l < h->n_lanes; ++l) off[l + 1] += off[l];
    const SnapBufs& sb = h->snap[h->parity];
    if (n > 0) {
        CK(cudaMemcpy(sb.a, a.data(), n * sizeof(RecA<Real>), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(sb.b, b.data(), n * sizeof(RecB), cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(sb.off, off.data(), off.size() * 4, cudaMemcpyHostToDevice));
    return MOSS_OK;
}

}  // namespace

// ============================================================================
namespace {

// lane setters (R25) for the lanes of scenario 0
template <typename Real>
void enqueue_set_lane(MossHandle* h, int n, int mode) {
    Ctx<Real> c = make_ctx<Real>(h, h->parity);
    k_set_lane<Real><<<(n + 255) / 256, 256, 0, h->stream>>>(c, n, h->d_lstage, h->d_lstage + n, mode);
}

int set_lane(MossHandle* h, int n, const int32_t* lane_ids, const int32_t* vals, int mode) {
    const int nl = h->scen_lane_off[1];
    if (n < 0 || (n > 0 && (!lane_ids || !vals)) || n > nl) return fail(h, MOSS_EINVAL, "bad arrays");
    for (int k = 0; k < n; ++k)
        if (lane_ids[k] < 0 || lane_ids[k] >= nl) return fail(h, MOSS_EINVAL, "lane id out of range");
    if (n == 0) return MOSS_OK;
    std::vector<int32_t> buf(2 * (size_t)n);
    for (int k = 0; k < n; ++k) { buf[k] = lane_ids[k]; buf[n + k] = vals[k]; }
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(h->d_lstage, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice));
    if (h->precision == 64) enqueue_set_lane<double>(h, n, mode);
    else enqueue_set_lane<float>(h, n, mode);
    CK(cudaGetLastError());
    for (int k = 0; k < n; ++k) {
        LaneInfo& li = h->lanes[lane_ids[k]];
        if (mode == 0) std::memcpy(&li.vmax, &vals[k], 4);
        else li.flags = vals[k] ? (li.flags | LF_RESTRICTED) : (li.flags & ~LF_RESTRICTED);
    }
    return MOSS_OK;
}

// road b is reachable from some lane of road a (the rule routes obey)
bool turn_from_some_lane(const MossHandle* h, int a, int b) {
    const int2 sp = h->road_span[a];
    for (int l = sp.x; l < sp.y; ++l)
        for (int j = h->lanes[l].jb; j < h->lanes[l].je; ++j)
            if (h->lanes[j].road == b) return true;
    return false;
}

template <typename Real>
int reroute_impl(MossHandle* h, int n, const int32_t* vids, const int32_t* route_off, const int32_t* roads) {
    const int nv0 = h->scen_veh_off[1], nr0 = h->scen_road_off[1];
    // device scratch for this call
    int32_t *d_v = nullptr, *d_lane = nullptr;
    int2* d_sp = nullptr;
    auto cleanup = [&]() {
        raw_free(h, d_v, n * 4); raw_free(h, d_lane, n * 4); raw_free(h, d_sp, n * sizeof(int2));
    };
    d_v = (int32_t*)raw_alloc(h, n * 4);
    d_lane = (int32_t*)raw_alloc(h, n * 4);
    d_sp = (int2*)raw_alloc(h, n * sizeof(int2));
    if (!d_v || !d_lane || !d_sp) {
        cleanup();
        return fail(h, MOSS_ENOMEM, "re-routing scratch");
    }
    Ctx<Real> c = make_ctx<Real>(h, h->parity);
    const int nb = (n + 255) / 256, grid = std::max(1, h->sm_count * 4);
    std::vector<int32_t> lane(n, -1), status(nv0);
    cudaError_t e = cudaMemcpy(d_v, vids, n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_lane, lane.data(), n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_mark_vehicles<<<nb, 256, 0, h->stream>>>(h->d_req, n, d_v, 1);
        k_find_lanes<Real><<<grid, 256, 0, h->stream>>>(c, h->d_req, d_lane);
        e = cudaStreamSynchronize(h->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpy(lane.data(), d_lane, n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(status.data(), h->d_vstatus, nv0 * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cleanup();
        return fail(h, MOSS_ECUDA, cudaGetErrorString(e));
    }
    // validate every request first (all or nothing)
    std::string why;
    std::vector<int> prev(n, -1);
    for (int k = 0; k < n && why.empty(); ++k) {
        const int g = vids[k], a = route_off[k], b = route_off[k + 1];
        if (status[g] == MOSS_ST_ARRIVED) { why = "vehicle has arrived"; break; }
        int first;
        if (status[g] == MOSS_ST_WAITING) {
            first = h->lanes[h->start_lane[g]].road;
        } else {
            const int l = lane[k];
            if (l < 0) { why = "active vehicle not found"; break; }
            first = h->lanes[l].road;  // a junction lane: the road it enters
            if (h->lanes[l].lo < 0) prev[k] = h->lane_src_road[l];
        }
        if (roads[a] != first) { why = "the route must start with the vehicle's road"; break; }
        for (int q = a; q + 1 < b; ++q)
            if (!turn_from_some_lane(h, roads[q], roads[q + 1])) { why = "roads not joined"; break; }
    }
    if (!why.empty()) {
        k_mark_vehicles<<<nb, 256, 0, h->stream>>>(h->d_req, n, d_v, 0);
        cudaStreamSynchronize(h->stream);
        cleanup();
        return fail(h, MOSS_EINVAL, why);
    }
    // append the routes (the road just left stays in front for a vehicle on
    // a junction lane)
    const size_t old = h->routes.size();
    std::vector<int2> sp(n);
    for (int k = 0; k < n; ++k) {
        const int beg = (int)h->routes.size();
        if (prev[k] >= 0) h->routes.push_back(prev[k]);
        for (int q = route_off[k]; q < route_off[k + 1]; ++q) h->routes.push_back(roads[q]);
        sp[k] = make_int2(beg, (int)h->routes.size());
    }
    if (h->routes.size() > h->routes_cap) {  // grow the device route buffer
        const size_t cap = std::max(h->routes.size(), 2 * h->routes_cap);
        int32_t* nr = (int32_t*)raw_alloc(h, cap * 4);
        if (!nr) {
            h->routes.resize(old);
            k_mark_vehicles<<<nb, 256, 0, h->stream>>>(h->d_req, n, d_v, 0);
            cudaStreamSynchronize(h->stream);
            cleanup();
            return fail(h, MOSS_ENOMEM, "route buffer");
        }
        cudaMemcpy(nr, h->d_routes, old * 4, cudaMemcpyDeviceToDevice);
        for (auto& a : h->allocs)
            if (a.first == (void*)h->d_routes) {
                raw_free(h, a.first, a.second);
                h->bytes += cap * 4 - a.second;
                a = std::make_pair((void*)nr, cap * 4);
            }
        h->d_routes = nr;
        h->routes_cap = cap;
        destroy_graphs(h);
        TRY(build_graphs(h));
        c = make_ctx<Real>(h, h->parity);
    }
    e = cudaMemcpy(h->d_routes + old, h->routes.data() + old, (h->routes.size() - old) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_sp, sp.data(), n * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_apply_routes<Real><<<grid, 256, 0, h->stream>>>(c, h->d_req, n, d_v, d_sp);
        k_mark_vehicles<<<nb, 256, 0, h->stream>>>(h->d_req, n, d_v, 0);
        e = cudaStreamSynchronize(h->stream);
    }
    cleanup();
    if (e != cudaSuccess) return fail(h, MOSS_ECUDA, cudaGetErrorString(e));
    for (int k = 0; k < n; ++k) h->route_span[vids[k]] = sp[k];
    (void)nr0;
    return check_device(h);
}

int reroute(MossHandle* h, int n, const int32_t* vids, const int32_t* route_off, const int32_t* roads) {
    const int nv0 = h->scen_veh_off[1], nr0 = h->scen_road_off[1];
    if (n < 0 || (n > 0 && (!vids || !route_off || !roads))) return fail(h, MOSS_EINVAL, "bad arrays");
    if (n == 0) return MOSS_OK;
    if (route_off[0] != 0) return fail(h, MOSS_EINVAL, "route_off[0] != 0");
    std::vector<char> seen(nv0, 0);
    for (int k = 0; k < n; ++k) {
        if (vids[k] < 0 || vids[k] >= nv0) return fail(h, MOSS_EINVAL, "vehicle id out of range");
        if (seen[vids[k]]++) return fail(h, MOSS_EINVAL, "a vehicle appears twice");
        if (route_off[k + 1] <= route_off[k]) return fail(h, MOSS_EINVAL, "every route needs a road");
        for (int q = route_off[k]; q < route_off[k + 1]; ++q)
            if (roads[q] < 0 || roads[q] >= nr0) return fail(h, MOSS_EINVAL, "road id out of range");
    }
    CK(cudaStreamSynchronize(h->stream));
    return h->precision == 64 ? reroute_impl<double>(h, n, vids, route_off, roads)
                              : reroute_impl<float>(h, n, vids, route_off, roads);
}

template <typename Real>
int scen_lane_metrics(MossHandle* h, int s, int32_t* queue, double* speed) {
    Ctx<Real> c = make_ctx<Real>(h, h->parity);
    if (queue) {
        const int l0 = h->scen_lane_off[s], l1 = h->scen_lane_off[s + 1];
        if (l1 > l0) {
            k_lane_queue<Real><<<(l1 - l0 + 255) / 256, 256, 0, h->stream>>>(c, l0, l1, (int32_t*)h->d_mbuf);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(queue, h->d_mbuf, (size_t)(l1 - l0) * 4, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
    }
    if (speed) {
        const int r0 = h->scen_road_off[s], r1 = h->scen_road_off[s + 1];
        if (r1 > r0) {
            k_road_speed<Real><<<(r1 - r0 + 255) / 256, 256, 0, h->stream>>>(c, r0, r1, (double*)h->d_mbuf);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(speed, h->d_mbuf, (size_t)(r1 - r0) * 8, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
    }
    return check_device(h);
}

int lane_metrics(MossHandle* h, int s, int32_t* queue, double* speed) {
    if (s < 0 || s >= h->n_scen) return fail(h, MOSS_EINVAL, "scenario index out of range");
    return h->precision == 64 ? scen_lane_metrics<double>(h, s, queue, speed)
                              : scen_lane_metrics<float>(h, s, queue, speed);
}

}  // namespace

extern "C" {

int moss_create(const MossNetwork* net, const MossVehicles* veh, const MossParams* prm,
                void* cuda_stream, moss_t* out) {
    return moss_batch_create(1, net, veh, prm, cuda_stream, out);
}

int moss_batch_create(int n, const MossNetwork* nets, const MossVehicles* vehs,
                      const MossParams* prms, void* cuda_stream, moss_t* out) {
    return moss_batch_create_with_allocator(n, nets, vehs, prms, cuda_stream, nullptr, out);
}

int moss_batch_create_with_allocator(int n, const MossNetwork* nets, const MossVehicles* vehs,
                                     const MossParams* prms, void* cuda_stream, const MossAllocator* allocator,
                                     moss_t* out) {
    if (!out) return MOSS_EINVAL;
    *out = nullptr;
    if (!nets || !vehs || !prms) return MOSS_EINVAL;
    if (allocator && (!allocator->alloc || !allocator->release)) return MOSS_EINVAL;
    MossHandle* h = new (std::nothrow) MossHandle();
    if (!h) return MOSS_ENOMEM;
    if (allocator) h->allocator = *allocator;
    int rc;
    try {
        rc = create_impl(n, nets, vehs, prms, cuda_stream, h);
    } catch (const std::bad_alloc&) {
        rc = fail(h, MOSS_ENOMEM, "host allocation failed");
    }
    if (rc != MOSS_OK) {
        fprintf(stderr, "moss_create: %s\n", h->err.c_str());
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return MOSS_OK;
}

int moss_step(moss_t h, int n) {
    if (!h) return MOSS_EINVAL;
    if (n < 0) return fail(h, MOSS_EINVAL, "negative step count");
    if (h->timing) {
        for (int k = 0; k < n; ++k) {
            enqueue(h, h->parity, true);
            h->parity ^= 1;
            CK(cudaEventSynchronize(h->ev[N_STEP_KERNELS]));
            // reported order: decide, lanescan, place, resolve
            static const int slot_of[N_STEP_KERNELS] = {0, 3, 1, 2};
            for (int q = 0; q < N_STEP_KERNELS; ++q) {
                float ms = 0;
                CK(cudaEventElapsedTime(&ms, h->ev[q], h->ev[q + 1]));
                h->kms[slot_of[q]] += ms;
            }
            h->ksteps++;
        }
        CK(cudaGetLastError());
        return MOSS_OK;
    }
    int k = 0;
    for (; k + 2 <= n; k += 2) CK(cudaGraphLaunch(h->g2[h->parity], h->stream));
    if (k < n) {
        CK(cudaGraphLaunch(h->g1[h->parity], h->stream));
        h->parity ^= 1;
    }
    return MOSS_OK;
}

int moss_set_signal_phase(moss_t h, int n, const int32_t* junction_ids, const int32_t* phase_idx) {
    return moss_batch_set_signal_phase(h, 0, n, junction_ids, phase_idx);
}

int moss_batch_set_signal_phase(moss_t h, int scenario, int n, const int32_t* junction_ids,
                                const int32_t* phase_idx) {
    if (!h) return MOSS_EINVAL;
    if (scenario < 0 || scenario >= h->n_scen) return fail(h, MOSS_EINVAL, "scenario out of range");
    if (n < 0 || (n > 0 && (!junction_ids || !phase_idx))) return fail(h, MOSS_EINVAL, "bad arrays");
    const int j0 = h->scen_junc_off[scenario], nj = h->scen_junc_off[scenario + 1] - j0;
    if (n > nj) return fail(h, MOSS_EINVAL, "more junctions than the scenario has");
    if (n == 0) return MOSS_OK;
    // the pinned staging area is reused: wait until the previous copy out of
    // it ran; then one pass checks and stages (nothing is enqueued on failure)
    CK(cudaEventSynchronize(h->stage_free));
    const int32_t* po = h->junc_phase_off.data() + j0;
    int32_t* sj = h->h_stage;
    int32_t* sp = h->h_stage + n;
    for (int k = 0; k < n; ++k) {
        const int j = junction_ids[k], p = phase_idx[k];
        if (j < 0 || j >= nj) return fail(h, MOSS_EINVAL, "junction id out of range");
        const int np = po[j + 1] - po[j];
        if (p < 0 || p >= std::max(np, 1)) return fail(h, MOSS_EINVAL, "phase index out of range");
        sj[k] = j0 + j;
        sp[k] = p;
    }
    CK(cudaMemcpyAsync(h->d_stage, h->h_stage, 2 * n * 4, cudaMemcpyHostToDevice, h->stream));
    CK(cudaEventRecord(h->stage_free, h->stream));
    if (h->precision == 64) enqueue_set_signal<double>(h, n, POL_MANUAL);
    else enqueue_set_signal<float>(h, n, POL_MANUAL);
    CK(cudaGetLastError());
    return MOSS_OK;
}

int moss_set_signal_policy(moss_t h, int n, const int32_t* junction_ids, int32_t policy) {
    if (!h) return MOSS_EINVAL;
    if (policy < 0 || policy > 3) return fail(h, MOSS_EINVAL, "unknown policy");
    const int nj = h->scen_junc_off[1];
    if (n < 0 || (n > 0 && !junction_ids) || n > nj) return fail(h, MOSS_EINVAL, "bad arrays");
    if (n == 0) return MOSS_OK;
    for (int k = 0; k < n; ++k)
        if (junction_ids[k] < 0 || junction_ids[k] >= nj) return fail(h, MOSS_EINVAL, "junction id out of range");
    CK(cudaEventSynchronize(h->stage_free));
    for (int k = 0; k < n; ++k) {
        h->h_stage[k] = junction_ids[k];
        h->h_stage[n + k] = 0;
    }
    CK(cudaMemcpyAsync(h->d_stage, h->h_stage, 2 * n * 4, cudaMemcpyHostToDevice, h->stream));
    CK(cudaEventRecord(h->stage_free, h->stream));
    if (h->precision == 64) enqueue_set_signal<double>(h, n, policy);
    else enqueue_set_signal<float>(h, n, policy);
    CK(cudaGetLastError());
    return MOSS_OK;
}

int moss_set_road_lane_plan(moss_t h, int n, const int32_t* road_ids, const int32_t* plan_idx) {
    if (!h) return MOSS_EINVAL;
    const int nr0 = h->scen_road_off[1];
    if (n < 0 || (n > 0 && (!road_ids || !plan_idx))) return fail(h, MOSS_EINVAL, "bad arrays");
    for (int k = 0; k < n; ++k) {
        if (road_ids[k] < 0 || road_ids[k] >= nr0) return fail(h, MOSS_EINVAL, "road id out of range");
        if (plan_idx[k] < 0 || plan_idx[k] > 7) return fail(h, MOSS_EINVAL, "plan index must be 0..7");
    }
    if (n == 0) return MOSS_OK;
    CK(cudaStreamSynchronize(h->stream));
    int32_t* d = (int32_t*)raw_alloc(h, 2 * (size_t)n * 4);
    if (!d) return fail(h, MOSS_ENOMEM, "plan setter scratch");
    cudaError_t e = cudaMemcpy(d, road_ids, n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + n, plan_idx, n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int nb = (n + 255) / 256, grid = std::max(1, h->sm_count * 4);
        if (h->precision == 64) {
            Ctx<double> c = make_ctx<double>(h, h->parity);
            k_set_plan<double><<<nb, 256, 0, h->stream>>>(c, n, d, d + n, h->d_jl_plans, h->d_road_mark);
            k_plan_next_lanes<double><<<grid, 256, 0, h->stream>>>(c, h->d_road_mark);
        } else {
            Ctx<float> c = make_ctx<float>(h, h->parity);
            k_set_plan<float><<<nb, 256, 0, h->stream>>>(c, n, d, d + n, h->d_jl_plans, h->d_road_mark);
            k_plan_next_lanes<float><<<grid, 256, 0, h->stream>>>(c, h->d_road_mark);
        }
        k_unmark_roads<<<nb, 256, 0, h->stream>>>(n, d, h->d_road_mark);
        e = cudaStreamSynchronize(h->stream);
    }
    raw_free(h, d, 2 * (size_t)n * 4);
    if (e != cudaSuccess) return fail(h, MOSS_ECUDA, cudaGetErrorString(e));
    for (int k = 0; k < n; ++k) {  // the host copy of the lane table
        const int2 sp = h->road_span[road_ids[k]];
        for (int l = sp.x; l < sp.y; ++l)
            for (int j = h->lanes[l].jb; j < h->lanes[l].je; ++j) {
                const bool on = (h->jl_plans[j] >> plan_idx[k]) & 1;
                h->lanes[j].flags = on ? (h->lanes[j].flags & ~LF_OFF) : (h->lanes[j].flags | LF_OFF);
            }
    }
    return check_device(h);
}

int moss_set_vehicle_route(moss_t h, int n, const int32_t* vehicle_ids, const int32_t* route_off,
                           const int32_t* roads) {
    if (!h) return MOSS_EINVAL;
    return reroute(h, n, vehicle_ids, route_off, roads);
}

int moss_set_lane_max_speed(moss_t h, int n, const int32_t* lane_ids, const float* vmax) {
    if (!h) return MOSS_EINVAL;
    if (n > 0 && !vmax) return fail(h, MOSS_EINVAL, "bad arrays");
    std::vector<int32_t> bits(std::max(n, 0));
    for (int k = 0; k < n; ++k) {
        if (!(vmax[k] > 0.0f) || !std::isfinite(vmax[k])) return fail(h, MOSS_EINVAL, "speed limit must be > 0");
        std::memcpy(&bits[k], &vmax[k], 4);
    }
    return set_lane(h, n, lane_ids, bits.data(), 0);
}

int moss_set_lane_restriction(moss_t h, int n, const int32_t* lane_ids, const int32_t* flags) {
    if (!h) return MOSS_EINVAL;
    return set_lane(h, n, lane_ids, flags, 1);
}

int moss_get_lane_queue(moss_t h, int32_t* queue) {
    if (!h) return MOSS_EINVAL;
    if (!queue) return fail(h, MOSS_EINVAL, "null output");
    return lane_metrics(h, 0, queue, nullptr);
}

int moss_get_road_speed(moss_t h, double* speed) {
    if (!h) return MOSS_EINVAL;
    if (!speed) return fail(h, MOSS_EINVAL, "null output");
    return lane_metrics(h, 0, nullptr, speed);
}

int moss_batch_get_lane_queue(moss_t h, int scenario, int32_t* queue) {
    if (!h) return MOSS_EINVAL;
    if (!queue) return fail(h, MOSS_EINVAL, "null output");
    return lane_metrics(h, scenario, queue, nullptr);
}

int moss_batch_get_road_speed(moss_t h, int scenario, double* speed) {
    if (!h) return MOSS_EINVAL;
    if (!speed) return fail(h, MOSS_EINVAL, "null output");
    return lane_metrics(h, scenario, nullptr, speed);
}

int moss_get_signal_state(moss_t h, int n, const int32_t* junction_ids, int32_t* phase, int32_t* elapsed,
                          int32_t* next_phase) {
    if (!h) return MOSS_EINVAL;
    if (h->n_scen != 1) return fail(h, MOSS_EINVAL, "signal state of batches is not available");
    if (n < 0 || (n > 0 && (!junction_ids || !phase || !elapsed || !next_phase)))
        return fail(h, MOSS_EINVAL, "bad arrays");
    const int nj = h->n_junctions;
    for (int k = 0; k < n; ++k)
        if (junction_ids[k] < 0 || junction_ids[k] >= nj) return fail(h, MOSS_EINVAL, "junction id out of range");
    if (n == 0) return MOSS_OK;
    CK(cudaStreamSynchronize(h->stream));
    std::vector<int32_t> st(nj), pol(nj);
    std::vector<int4> mp(nj);
    CK(cudaMemcpy(st.data(), h->d_junc_state, nj * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(pol.data(), h->d_junc_policy, nj * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(mp.data(), h->d_mp, nj * sizeof(int4), cudaMemcpyDeviceToHost));
    for (int k = 0; k < n; ++k) {
        const int j = junction_ids[k], x = st[j];
        phase[k] = (x & 512) ? -1 : (x & 15);
        next_phase[k] = (x & 512) || !(x & 256) ? -1 : ((x >> 10) & 15);
        elapsed[k] = pol[j] == POL_MAXP ? mp[j].y : 0;
    }
    return check_device(h);
}

int moss_get_metrics(moss_t h, MossMetrics* out) {
    if (!h) return MOSS_EINVAL;
    return scen_metrics(h, 0, out);
}

int moss_batch_get_metrics(moss_t h, int scenario, MossMetrics* out) {
    if (!h) return MOSS_EINVAL;
    return scen_metrics(h, scenario, out);
}

int moss_metrics_enqueue(moss_t h, int scenario, int slot) {
    if (!h) return MOSS_EINVAL;
    if (scenario < 0 || scenario >= h->n_scen) return fail(h, MOSS_EINVAL, "scenario index out of range");
    if (slot < 0 || slot >= MOSS_METRIC_SLOTS) return fail(h, MOSS_EINVAL, "metric slot out of range");
    // a slot still in flight is waited for before its memory is reused
    if (h->rb_pending[slot]) CK(cudaEventSynchronize(h->rb_ev[slot]));
    TRY(enqueue_readback(h, scenario, slot));
    CK(cudaEventRecord(h->rb_ev[slot], h->stream));
    h->rb_pending[slot] = true;
    h->rb_scen[slot] = scenario;
    return MOSS_OK;
}

int moss_metrics_read(moss_t h, int slot, MossMetrics* out) {
    if (!h) return MOSS_EINVAL;
    if (!out) return fail(h, MOSS_EINVAL, "null output");
    if (slot < 0 || slot >= MOSS_METRIC_SLOTS) return fail(h, MOSS_EINVAL, "metric slot out of range");
    if (!h->rb_pending[slot]) return fail(h, MOSS_EINVAL, "nothing enqueued in this metric slot");
    CK(cudaEventSynchronize(h->rb_ev[slot]));
    h->rb_pending[slot] = false;
    return readback_metrics(h, h->rb_scen[slot], slot, out);
}

int moss_get_state(moss_t h, MossState* out) {
    if (!h) return MOSS_EINVAL;
    if (h->n_scen != 1) return fail(h, MOSS_EINVAL, "use moss_batch_get_state for batches");
    return scen_state(h, 0, out);
}

int moss_batch_get_state(moss_t h, int scenario, MossState* out) {
    if (!h) return MOSS_EINVAL;
    return scen_state(h, scenario, out);
}

int moss_set_state(moss_t h, const MossState* in, int64_t step) {
    if (!h) return MOSS_EINVAL;
    if (h->n_scen != 1) return fail(h, MOSS_EINVAL, "moss_set_state takes single-scenario handles");
    if (!in || !in->status || !in->lane || !in->s || !in->v || !in->rc)
        return fail(h, MOSS_EINVAL, "null state array");
    if (step < 0) return fail(h, MOSS_EINVAL, "negative step");
    CK(cudaStreamSynchronize(h->stream));
    const int NV = h->n_veh;
    std::vector<int> order;
    std::vector<double> s(NV), v(NV);
    std::vector<int> lane_of(NV, -1), rc(NV, 0);
    long long n_act = 0, n_arr = 0;
    for (int i = 0; i < NV; ++i) {
        const int st = in->status[i];
        if (st < 0 || st > 2) return fail(h, MOSS_EINVAL, "bad status");
        s[i] = in->s[i]; v[i] = in->v[i]; rc[i] = in->rc[i];
        if (st == MOSS_ST_ARRIVED) n_arr++;
        if (st != MOSS_ST_ACTIVE) continue;
        n_act++;
        const int l = in->lane[i];
        const int nr = h->route_span[i].y - h->route_span[i].x;
        if (l < 0 || l >= h->n_lanes) return fail(h, MOSS_EINVAL, "active vehicle on a bad lane");
        if (rc[i] < 0 || rc[i] >= nr) return fail(h, MOSS_EINVAL, "route cursor out of range");
        const int road = h->routes[h->route_span[i].x + rc[i]];
        if (h->lanes[l].lo >= 0) {
            if (h->lanes[l].road != road) return fail(h, MOSS_EINVAL, "lane is not on the route's road");
        } else {
            if (rc[i] + 1 >= nr || h->lane_src_road[l] != road ||
                h->lanes[l].road != h->routes[h->route_span[i].x + rc[i] + 1])
                return fail(h, MOSS_EINVAL, "junction lane does not join the route's roads");
        }
        if (!(s[i] >= 0.0 && s[i] <= h->lanes[l].L) || !(v[i] >= 0.0) || !std::isfinite(v[i]))
            return fail(h, MOSS_EINVAL, "position or speed out of range");
        lane_of[i] = l;
        order.push_back(i);
    }
    // departure queues: waiting vehicles must be each queue's tail
    std::vector<int32_t> qh(h->n_lanes);
    for (int l = 0; l < h->n_lanes; ++l) {
        int k = h->q_off[l];
        while (k < h->q_off[l + 1] && in->status[h->q_ids[k]] != MOSS_ST_WAITING) ++k;
        qh[l] = k;
        for (int q = k; q < h->q_off[l + 1]; ++q)
            if (in->status[h->q_ids[q]] != MOSS_ST_WAITING)
                return fail(h, MOSS_EINVAL, "waiting vehicles must form the tail of their start lane's queue");
    }
    // lane-major snapshot order: (lane, s desc, id asc), s rounded to the precision
    std::vector<double> key(NV);
    for (int i : order) key[i] = h->precision == 64 ? s[i] : (double)(float)s[i];
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        if (lane_of[a] != lane_of[b]) return lane_of[a] < lane_of[b];
        if (key[a] != key[b]) return key[a] > key[b];
        return a < b;
    });
    int rc2 = h->precision == 64 ? upload_state<double>(h, order, s, v, lane_of, rc)
                                 : upload_state<float>(h, order, s, v, lane_of, rc);
    if (rc2) return rc2;
    std::vector<int32_t> status(in->status, in->status + NV);
    CK(cudaMemcpy(h->d_vstatus, status.data(), NV * 4, cudaMemcpyHostToDevice));
    CK(cudaMemset(h->d_vflags, 0, NV * 4));
    CK(cudaMemcpy(h->d_q_head, qh.data(), qh.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_step, &step, sizeof(long long), cudaMemcpyHostToDevice));
    long long cur[2] = {n_act, n_arr};
    CK(cudaMemcpy(h->d_metrics + M_CUR_ACTIVE, cur, sizeof(cur), cudaMemcpyHostToDevice));
    Counters c{};
    CK(cudaMemcpy(&c, h->d_cnt + h->parity, sizeof(c), cudaMemcpyDeviceToHost));
    c.n_cur = (int)n_act; c.n_ent = 0; c.n_cand = 0; c.ticket_lane = 0; c.res_done = 0;
    CK(cudaMemcpy(h->d_cnt + h->parity, &c, sizeof(c), cudaMemcpyHostToDevice));
    TRY(junction_init(h));
    CK(cudaStreamSynchronize(h->stream));
    return MOSS_OK;
}

int moss_synchronize(moss_t h) {
    if (!h) return MOSS_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    return check_device(h);
}

int moss_device_bytes(moss_t h, size_t* out) {
    if (!h || !out) return MOSS_EINVAL;
    *out = h->bytes;
    return MOSS_OK;
}

int moss_batch_size(moss_t h, int* out) {
    if (!h || !out) return MOSS_EINVAL;
    *out = h->n_scen;
    return MOSS_OK;
}

void moss_destroy(moss_t h) {
    if (!h) return;
    free_all(h);
    delete h;
}

const char* moss_last_error(moss_t h) {
    if (!h) return "null handle";
    return h->err.c_str();
}

int moss_set_kernel_timing(moss_t h, int enable) {
    if (!h) return MOSS_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    h->timing = enable != 0;
    for (double& x : h->kms) x = 0;
    h->ksteps = 0;
    return MOSS_OK;
}

// time `steps` steps (the simulation advances normally) with the current
// launch configuration; returns the summed kernel milliseconds
static int time_steps(MossHandle* h, int steps, double* ms) {
    double tot = 0;
    for (int k = 0; k < steps; ++k) {
        enqueue(h, h->parity, true);
        h->parity ^= 1;
        CK(cudaEventSynchronize(h->ev[N_STEP_KERNELS]));
        float x = 0;
        CK(cudaEventElapsedTime(&x, h->ev[0], h->ev[N_STEP_KERNELS]));
        tot += x;
    }
    CK(cudaGetLastError());
    *ms = tot;
    return MOSS_OK;
}

int moss_autotune(moss_t h, int trial_steps, int* chosen3) {
    if (!h) return MOSS_EINVAL;
    if (trial_steps < 1) return fail(h, MOSS_EINVAL, "trial_steps must be >= 1");
    CK(cudaStreamSynchronize(h->stream));
    // coordinate search over blocks per SM of each kernel; results do not
    // depend on the launch configuration, only the time does
    static const int cand_decide[] = {3, 4, 5};
    static const int cand_lanescan[] = {1, 2, 4};
    static const int cand_place[] = {4, 8, 16};
    const int* cands[3] = {cand_decide, cand_lanescan, cand_place};
    int* knobs[3] = {&h->cfg_decide, &h->cfg_lanescan, &h->cfg_place};
    for (int d = 0; d < 3; ++d) {
        int best = *knobs[d];
        double best_ms = 1e300;
        for (int k = 0; k < 3; ++k) {
            *knobs[d] = cands[d][k];
            double ms = 0;
            TRY(time_steps(h, trial_steps, &ms));
            if (ms < best_ms) { best_ms = ms; best = cands[d][k]; }
        }
        *knobs[d] = best;
    }
    destroy_graphs(h);
    TRY(build_graphs(h));
    if (chosen3) { chosen3[0] = h->cfg_decide; chosen3[1] = h->cfg_lanescan; chosen3[2] = h->cfg_place; }
    return check_device(h);
}

int moss_selftest_bounded_wait(void* cuda_stream) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    void* buf = nullptr;
    if (cudaMalloc(&buf, 64) != cudaSuccess) { cudaGetLastError(); return MOSS_ECUDA; }
    int rc = MOSS_OK;
    int err = 0;
    if (cudaMemsetAsync(buf, 0, 64, st) != cudaSuccess) rc = MOSS_ECUDA;
    if (rc == MOSS_OK) {
        k_selftest_wait<<<1, 32, 0, st>>>((unsigned long long*)buf, (int*)((char*)buf + 32));
        if (cudaGetLastError() != cudaSuccess) rc = MOSS_ECUDA;
    }
    if (rc == MOSS_OK && cudaMemcpyAsync(&err, (char*)buf + 32, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = MOSS_ECUDA;
    if (rc == MOSS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = MOSS_ECUDA;
    cudaFree(buf);
    if (rc != MOSS_OK) return rc;
    return (err & ERR_TIMEOUT) ? MOSS_ETIMEOUT : MOSS_EDEVICE;
}

int moss_kernel_times(moss_t h, double* ms4, int64_t* steps) {
    if (!h || !ms4 || !steps) return MOSS_EINVAL;
    for (int k = 0; k < 4; ++k) ms4[k] = h->kms[k];
    *steps = h->ksteps;
    return MOSS_OK;
}

}  // extern "C"
