// Host side of the C ABI declared in include/moss.h: input validation, the
// union network of a batch, device buffers, CUDA-graph replay of the step
// kernels, and state / metric transfer.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <thread>
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

// a slot of a slot batch: first index and capacity of its lanes, roads,
// junctions, phases, junction-lane entries (jj), vehicles, route entries and
// start-lane entries (SO, one per lane)
struct SlotInfo {
    int LO = 0, nl_cap = 0, RO = 0, nr_cap = 0, JO = 0, nj_cap = 0, PO = 0, np_cap = 0;
    int JJ = 0, njj_cap = 0, VO = 0, nv_cap = 0, QO = 0, nq_cap = 0, SO = 0;
    bool loaded = false, retired = false;
    long long retire_step = 0;  // steps enqueued when it was retired
};

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
    std::vector<int> scen_nv, scen_nl, scen_nj, scen_nr;  // vehicles, lanes, junctions, roads in use per scenario
    std::vector<int32_t> junc_offset, phase_green, phase_amber;
    std::vector<int32_t> jj_off, jj_lane, jj_from;  // junction lanes grouped by junction (CSR)
    std::vector<int32_t> q_head;                     // initial departure-queue heads
    bool slots = false;                              // a slot batch (moss_slots_create)
    char* h_load = nullptr;                          // pinned staging of slot loads
    size_t load_cap = 0;
    cudaEvent_t load_free = nullptr;                 // recorded after the last copy out of h_load
    std::vector<SlotInfo> slot;
    long long steps_enqueued = 0;
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
    std::vector<int4> scen_lanes;     // [n_scen] first lane, first junction lane, end of the lanes in use
    int32_t* d_lstage = nullptr;      // setter arguments for lanes (2 * n_lanes)
    void* d_mbuf = nullptr;           // metric output (max(n_lanes, n_roads) doubles)
    int2* d_route_span = nullptr;
    int32_t *d_routes = nullptr, *d_dep = nullptr, *d_vstatus = nullptr,
            *d_vflags = nullptr;
    int32_t *d_q_off = nullptr, *d_q_ids = nullptr, *d_q_head = nullptr, *d_start_lanes = nullptr;
    uint32_t *d_key0 = nullptr, *d_key1 = nullptr;
    int4* d_scen_lanes = nullptr;
    int4* d_runstat = nullptr;  // [RUNSTAT_MAX] k_decide run statistics for the run-weight fit
    int32_t* d_veh_base = nullptr;
    long long *d_step = nullptr, *d_metrics = nullptr;
    int32_t* d_scen_ctl = nullptr;    // per scenario: SC_FROZEN / SC_RETIRE
    long long* d_stop_at = nullptr;   // per scenario: step at which it freezes (-1: never)
    SnapBufs snap[2]{};
    int8_t* d_code = nullptr;
    void* d_stay = nullptr;  // SV<Real>[cap]
    void* d_ea = nullptr;    // RecA<Real>[cap]
    RecB* d_eb = nullptr;
    int32_t *d_enext = nullptr, *d_enter = nullptr, *d_leave = nullptr, *d_cand_late = nullptr;
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
    int cfg_runw = 0;    // weight of a road-lane slot in k_decide's runs (0: fitted each step)
    int cfg_lsr = 4;     // rounds of 128 lanes per warp in a lane-scan tile (4 or 2)
    int cfg_ccap = 256;  // lane-change candidates a k_decide block resolves itself

    int parity = 0;  // snapshot buffer holding the current step
    int step_mode = 0;               // 0: three kernels per step; 1: one cooperative launch
    unsigned* d_bar = nullptr;       // grid barrier of the cooperative step (count, generation)
    cudaError_t launch_err = cudaSuccess;
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

// fn(i0, i1) over [0, n) in contiguous chunks on the host's threads (large n)
template <typename F>
void parallel_for(long long n, F fn) {
    const int hw = (int)std::thread::hardware_concurrency();
    const int T = n < (1 << 16) ? 1 : std::max(1, std::min(hw, 32));
    if (T == 1) { fn(0ll, n); return; }
    std::vector<std::thread> th;
    const long long per = (n + T - 1) / T;
    for (int t = 0; t < T; ++t) {
        const long long a = t * per, b = std::min(n, a + per);
        if (a < b) th.emplace_back([=] { fn(a, b); });
    }
    for (auto& x : th) x.join();
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
    // (a flat CSR: the route check below is the hot loop of validation)
    std::vector<int32_t> ro_off(R + 1, 0), ro;
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
        ro.insert(ro.end(), common.begin(), common.end());
        ro_off[r + 1] = (int32_t)ro.size();
    }
    (void)road_out;
    const int N = veh->n;
    if (N < 0 || N >= (1 << 30)) return fail(h, MOSS_EINVAL, "vehicle count out of range");
    if (N > 0 && (!veh->route_off || !veh->routes || !veh->start_lane || !veh->dep || !veh->v0f))
        return fail(h, MOSS_EINVAL, "missing vehicle array");
    if (N > 0 && veh->route_off[0] != 0) return fail(h, MOSS_EINVAL, "route_off[0] != 0");
    // the vehicles in parallel chunks; the first failing vehicle is reported
    // (code 1..6 of the checks below)
    auto check = [&](int i) -> int {
        const int a = veh->route_off[i], b = veh->route_off[i + 1];
        if (b <= a) return 1;
        for (int k = a; k < b; ++k)
            if (veh->routes[k] < 0 || veh->routes[k] >= R) return 2;
        for (int k = a; k + 1 < b; ++k) {
            const int32_t* ob = ro.data() + ro_off[veh->routes[k]];
            const int32_t* oe = ro.data() + ro_off[veh->routes[k] + 1];
            if (!std::binary_search(ob, oe, veh->routes[k + 1])) return 3;
        }
        const int sl = veh->start_lane[i];
        if (sl < 0 || sl >= NRL || road_of[sl] != veh->routes[a]) return 4;
        if (veh->dep[i] < 0) return 5;
        if (!(veh->v0f[i] > 0.f) || !std::isfinite(veh->v0f[i])) return 6;
        return 0;
    };
    std::atomic<long long> bad{(long long)N};
    parallel_for(N, [&](long long i0, long long i1) {
        for (long long i = i0; i < i1 && i < bad.load(std::memory_order_relaxed); ++i)
            if (check((int)i)) {
                long long cur = bad.load();
                while (i < cur && !bad.compare_exchange_weak(cur, i)) {}
                return;
            }
    });
    if (bad.load() < N) {
        const int i = (int)bad.load();
        switch (check(i)) {
            case 1: return fail(h, MOSS_EINVAL, "every route needs at least one road");
            case 2: return fail(h, MOSS_EINVAL, "route road out of range");
            case 3: return fail(h, MOSS_EINVAL, "route of vehicle " + std::to_string(i) +
                                                    " uses a turn no lane of the road has");
            case 4: return fail(h, MOSS_EINVAL, "start lane must be a lane of the first road");
            case 5: return fail(h, MOSS_EINVAL, "negative departure step");
            default: return fail(h, MOSS_EINVAL, "v0f must be > 0");
        }
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

// lane-scan tiles of a step with `rounds` rounds of 128 lanes per warp
int lane_tiles(const MossHandle* h, int rounds) {
    const int tile = LANESCAN_THREADS * 4 * rounds;
    return (h->n_lanes + tile - 1) / tile;
}

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
    c.scen_lanes = h->d_scen_lanes;
    c.scen_ctl = h->d_scen_ctl; c.stop_at = h->d_stop_at;
    c.metrics = h->d_metrics;
    for (int k = 0; k < 2; ++k) {
        const SnapBufs& b = h->snap[k == 0 ? cur : 1 - cur];
        Snap<Real>& s = k == 0 ? c.cur : c.nxt;
        s.a = (RecA<Real>*)b.a; s.b = b.b; s.off = b.off;
    }
    c.code = h->d_code; c.stay = (SV<Real>*)h->d_stay;
    c.ea = (RecA<Real>*)h->d_ea; c.eb = h->d_eb; c.enext = h->d_enext; c.head = h->d_head;
    c.enter = h->d_enter; c.leave = h->d_leave; c.lane_tiles = h->d_lane_tiles;
    c.cand_late = h->d_cand_late;
    c.cands = (Cand<Real>*)h->d_cands; c.gap_head = h->d_gap_head;
    c.n_lane_tiles = lane_tiles(h, h->cfg_lsr); c.max_slot_tiles = h->max_slot_tiles;
    c.run_w = h->cfg_runw;
    c.runstat = h->d_runstat;
    c.cand_cap = h->cfg_ccap;
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
    // the lane scan's tickets, plus (MOSS_FOLD_RESOLVE) the candidate and
    // max-pressure chunks in front of them: their number is known on the
    // device only, so the grid takes every resident block it may need
    const int tickets = 1 + lane_tiles(h, h->cfg_lsr) + h->n_junc_chunks + (MOSS_FOLD_RESOLVE ? (h->n_jj + TILE - 1) / TILE + 8 : 0);
    g.lanescan = std::max(1, std::min(tickets, h->sm_count * h->cfg_lanescan));
    g.place = std::max(1, std::min(2 * h->max_slot_tiles, h->sm_count * h->cfg_place));
    return g;
}

// the step as one cooperative launch (moss_set_step_mode 1): every block of
// the grid resident, one per SM slot the occupancy allows
template <typename Real, bool Groups>
cudaError_t launch_coop(MossHandle* h, Ctx<Real>& c) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_coop<Real, Groups>, TILE, 0);
    if (e != cudaSuccess) return e;
    int grid = std::max(1, per_sm) * h->sm_count;
    int n_work = std::max(1, std::min(h->max_slot_tiles, grid));
    const int ns = (int)h->start_lanes.size();
    int n_ins = ns > 0 ? (ns + TILE - 1) / TILE : 0;
    unsigned* bar = h->d_bar;
    void* args[] = {(void*)&c, (void*)&n_work, (void*)&n_ins, (void*)&bar};
    return cudaLaunchCooperativeKernel((const void*)k_step_coop<Real, Groups>, grid, TILE, args, 0, h->stream);
}

template <typename Real>
void enqueue_step(MossHandle* h, int cur, bool timed) {
    Ctx<Real> c = make_ctx<Real>(h, cur);
    const Grids g = grids(h);
    cudaStream_t s = h->stream;
    if (timed) cudaEventRecord(h->ev[0], s);
    if (h->step_mode == 1) {
        c.n_lane_tiles = lane_tiles(h, 4);  // the single-launch step scans with the default tile
        const cudaError_t e = h->lane_groups ? launch_coop<Real, true>(h, c) : launch_coop<Real, false>(h, c);
        if (e != cudaSuccess) h->launch_err = e;
        if (timed)
            for (int q = 1; q <= N_STEP_KERNELS; ++q) cudaEventRecord(h->ev[q], s);
        return;
    }
    if (h->lane_groups) k_decide<Real, true><<<g.decide_work + g.decide_ins, TILE, 0, s>>>(c, g.decide_work);
    else k_decide<Real, false><<<g.decide_work + g.decide_ins, TILE, 0, s>>>(c, g.decide_work);
    if (timed) cudaEventRecord(h->ev[1], s);
#if !MOSS_FOLD_RESOLVE
    k_resolve<Real><<<g.resolve, TILE, 0, s>>>(c);
#endif
    if (timed) cudaEventRecord(h->ev[2], s);
    if (h->cfg_lsr == 2) k_lanescan<Real, 2><<<g.lanescan, LANESCAN_THREADS, 0, s>>>(c);
    else k_lanescan<Real, 4><<<g.lanescan, LANESCAN_THREADS, 0, s>>>(c);
    if (timed) cudaEventRecord(h->ev[3], s);
    k_place<Real><<<g.place, TILE, 0, s>>>(c);
    if (timed) cudaEventRecord(h->ev[4], s);
}

void enqueue(MossHandle* h, int cur, bool timed) {
    if (h->precision == 64) enqueue_step<double>(h, cur, timed);
    else enqueue_step<float>(h, cur, timed);
}

template <typename Real>
void enqueue_junction_init(MossHandle* h, int j0, int j1) {
    Ctx<Real> c = make_ctx<Real>(h, h->parity);
    const int nb = std::max(1, std::min((j1 - j0 + 255) / 256, h->sm_count * 4));
    k_junction_init<Real><<<nb, 256, 0, h->stream>>>(c, j0, j1);
}

// signal states of the current step of junctions [j0, j1)
int junction_init(MossHandle* h, int j0, int j1) {
    if (j1 <= j0) return MOSS_OK;
    if (h->precision == 64) enqueue_junction_init<double>(h, j0, j1);
    else enqueue_junction_init<float>(h, j0, j1);
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
            h->launch_err = cudaSuccess;
            for (int k = 0; k < nsteps; ++k) enqueue(h, (p + k) & 1, false);
            CK(cudaStreamEndCapture(h->stream, &g));
            if (h->launch_err != cudaSuccess) {
                cudaGraphDestroy(g);
                return cuda_fail(h, h->launch_err, "cooperative step launch");
            }
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

// the host tables of scenario k written at the given bases (first lane,
// junction, vehicle, road, phase and route entry of the scenario)
void fill_scenario(MossHandle* h, int k, const MossNetwork& nt, const MossVehicles& vh, const MossParams& pr,
                   int LO, int JO, int VO, int RO, int PO, int ROFF) {
    const int NRL = nt.n_road_lanes;
    h->scen_lanes[k] = make_int4(LO, LO + NRL, LO + nt.n_lanes, 0);
    std::vector<int32_t> road_of(NRL);
    for (int r = 0; r < nt.n_roads; ++r)
        for (int l = nt.road_lane_off[r]; l < nt.road_lane_off[r + 1]; ++l) road_of[l] = r;
    for (int l = 0; l < nt.n_lanes; ++l) {
        LaneInfo& li = h->lanes[LO + l];
        li.scen = k;
        li.flags = 0;
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
        h->lane_src_road[LO + l] = -1;
        h->jl_plans[LO + l] = 0xff;
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
        h->junc_offset[JO + j] = nt.junc_offset[j];
        h->junc_phase_off[JO + j] = PO + nt.junc_phase_off[j];
    }
    const int nph = nt.n_junctions ? nt.junc_phase_off[nt.n_junctions] : 0;
    for (int q = 0; q < nph; ++q) {
        h->phase_green[PO + q] = nt.phase_green[q];
        h->phase_amber[PO + q] = nt.phase_amber[q];
    }
    parallel_for(vh.n, [&](long long i0, long long i1) {
        for (long long i = i0; i < i1; ++i) {
            const int g = VO + (int)i;
            const int a = vh.route_off[i], b = vh.route_off[i + 1];
            for (int q = a; q < b; ++q) h->routes[ROFF + q] = RO + vh.routes[q];
            h->route_span[g] = make_int2(ROFF + a, ROFF + b);
            h->dep[g] = vh.dep[i];
            h->start_lane[g] = LO + vh.start_lane[i];
            h->v0f[g] = vh.v0f[i];
            h->veh_scen[g] = k;
        }
    });
    h->key0[k] = (uint32_t)(pr.seed & 0xffffffffull);
    h->key1[k] = (uint32_t)(pr.seed >> 32) ^ pr.scenario;
}

// network of a road with a turn that not all of its lanes serve (R27)
bool has_lane_groups(const MossHandle* h, int r0, int r1) {
    for (int r = r0; r < r1; ++r) {
        const int2 sp = h->road_span[r];
        std::vector<int> first;
        for (int l = sp.x; l < sp.y; ++l) {
            std::vector<int> outs;
            for (int j = h->lanes[l].jb; j < h->lanes[l].je; ++j) outs.push_back(h->lanes[j].road);
            std::sort(outs.begin(), outs.end());
            if (l == sp.x) first = outs;
            else if (outs != first) return true;
        }
    }
    return false;
}

// departure queues of the vehicles [v0, v1) on the lanes [l0, l1): the CSR
// q_off[l0 .. l1] from q_base on, ordered by (dep, id) (R18); every lane
// after the last one with vehicles is empty, the last lane's range ends at
// q_end (entries past the vehicles are never reached: q_head starts there)
void build_queues(MossHandle* h, int l0, int l1, int v0, int v1, int q_base, int q_end) {
    for (int l = l0; l <= l1; ++l) h->q_off[l] = 0;
    for (int i = v0; i < v1; ++i) h->q_off[h->start_lane[i] + 1]++;
    h->q_off[l0] = q_base;
    for (int l = l0; l < l1; ++l) h->q_off[l + 1] += h->q_off[l];
    std::vector<int32_t> fill(h->q_off.begin() + l0, h->q_off.begin() + l1);
    for (int i = v0; i < v1; ++i) h->q_ids[fill[h->start_lane[i] - l0]++] = i;
    for (int l = l0; l < l1; ++l) {
        std::stable_sort(h->q_ids.begin() + h->q_off[l], h->q_ids.begin() + h->q_off[l + 1],
                         [&](int a, int b) { return h->dep[a] < h->dep[b]; });
        h->q_head[l] = h->q_off[l];
    }
    // entries past the vehicles belong to the last lane (a padding lane of a
    // slot, with no vehicles of its own) and are never reached: its queue
    // head starts at their end
    if (q_end > h->q_off[l1]) {
        for (int q = h->q_off[l1]; q < q_end; ++q) h->q_ids[q] = q_base;
        h->q_head[l1 - 1] = q_end;
    }
    h->q_off[l1] = q_end;
}

// junction lanes of the junctions [j0, j1) (lanes [l0, l1)) grouped by
// junction from jj_base on, with the road lane each one leaves (the
// pressures of the max-pressure policy); the last junction's range ends at
// jj_end (padding entries name lane pad, a road lane, which adds nothing)
void build_jj(MossHandle* h, int j0, int j1, int l0, int l1, int jj_base, int jj_end, int pad) {
    for (int j = j0; j <= j1; ++j) h->jj_off[j] = 0;
    std::vector<int32_t> from(l1 - l0, -1);
    for (int l = l0; l < l1; ++l)
        if (h->lanes[l].lo >= 0)
            for (int q = h->lanes[l].jb; q < h->lanes[l].je; ++q) from[q - l0] = l;
    for (int l = l0; l < l1; ++l)
        if (h->lanes[l].lo < 0) h->jj_off[h->lanes[l].jb + 1]++;
    h->jj_off[j0] = jj_base;
    for (int j = j0; j < j1; ++j) h->jj_off[j + 1] += h->jj_off[j];
    std::vector<int32_t> fill(h->jj_off.begin() + j0, h->jj_off.begin() + j1);
    for (int l = l0; l < l1; ++l)
        if (h->lanes[l].lo < 0) {
            const int q = fill[h->lanes[l].jb - j0]++;
            h->jj_lane[q] = l;
            h->jj_from[q] = from[l - l0];
        }
    for (int q = h->jj_off[j1]; q < jj_end; ++q) { h->jj_lane[q] = pad; h->jj_from[q] = pad; }
    h->jj_off[j1] = jj_end;
}

// device buffers and graphs for the host tables of h (shared by batches and
// slot batches)
int device_setup(MossHandle* h, void* stream) {
    const int NL = h->n_lanes, NJ = h->n_junctions, NV = h->n_veh, n = h->n_scen;
    const long long tot_roads = (long long)h->road_span.size();
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
        junc[j].offset = h->junc_offset[j];
        junc[j].phase_off = h->junc_phase_off[j];
        junc[j].np = h->junc_phase_off[j + 1] - h->junc_phase_off[j];
        junc[j].scen = h->junc_scen[j];
    }
    // a slot's padding junction holds its spare phases but has no signal
    for (const SlotInfo& si : h->slot) junc[si.JO + si.nj_cap - 1].np = 0;
    TRY(upload(h, &h->d_junc, junc));
    TRY(upload(h, &h->d_phase_green, h->phase_green));
    TRY(upload(h, &h->d_phase_amber, h->phase_amber));
    TRY(upload(h, &h->d_junc_policy, std::vector<int32_t>(NJ, POL_FIXED)));
    TRY(upload(h, &h->d_junc_manual, std::vector<int32_t>(NJ, 0)));
    TRY(dalloc(h, &h->d_junc_state, NJ));
    TRY(upload(h, &h->d_jj_off, h->jj_off));
    {
        std::vector<int32_t> a(h->jj_lane), b(h->jj_from);
        if (a.empty()) { a.push_back(0); b.push_back(0); }
        TRY(upload(h, &h->d_jj_lane, a));
        TRY(upload(h, &h->d_jj_from, b));
    }
    h->n_jj = h->jj_off[NJ];
    TRY(upload(h, &h->d_mp, std::vector<int4>(std::max(NJ, 1), make_int4(0, 1, -1, 0))));
    TRY(upload(h, &h->d_mp_press, std::vector<int32_t>((size_t)std::max(NJ, 1) * 8, 0)));
    {
        std::vector<int2> span(h->road_span);
        if (span.empty()) span.push_back(make_int2(0, 0));
        TRY(upload(h, &h->d_road_span, span));
    }
    TRY(dalloc(h, &h->d_lstage, 2 * (size_t)std::max(NL, 1)));
    TRY(upload(h, &h->d_jl_plans, h->jl_plans.empty() ? std::vector<int32_t>(1, 0xff) : h->jl_plans));
    TRY(upload(h, &h->d_road_mark, std::vector<int8_t>(std::max<long long>(tot_roads, 1), 0)));
    TRY(dalloc(h, (char**)&h->d_mbuf, sizeof(double) * (size_t)std::max(std::max(NL, (int)tot_roads), 1)));
    {
        std::vector<int2> span(h->route_span);
        if (span.empty()) span.push_back(make_int2(0, 0));
        TRY(upload(h, &h->d_route_span, span));
        // room for re-routed vehicles' routes (grown on demand)
        if (!h->slots) h->routes_cap = h->routes.size() + std::max<size_t>(h->routes.size() / 4, 1 << 16);
        else h->routes_cap = std::max<size_t>(h->routes.size(), 1);
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
    TRY(upload(h, &h->d_q_head, h->q_head));
    TRY(upload(h, &h->d_start_lanes, h->start_lanes));
    TRY(upload(h, &h->d_key0, h->key0));
    TRY(upload(h, &h->d_key1, h->key1));
    TRY(upload(h, &h->d_scen_lanes, h->scen_lanes));
    TRY(upload(h, &h->d_runstat, std::vector<int4>(RUNSTAT_MAX, make_int4(0, 0, 0, 0))));
    TRY(upload(h, &h->d_veh_base, std::vector<int32_t>(h->scen_veh_off.begin(), h->scen_veh_off.end() - 1)));
    TRY(upload(h, &h->d_step, std::vector<long long>(n, 0)));
    TRY(upload(h, &h->d_metrics, std::vector<long long>((size_t)n * M_NFIELDS, 0)));
    TRY(upload(h, &h->d_scen_ctl, std::vector<int32_t>(n, h->slots ? SC_FROZEN : 0)));
    TRY(upload(h, &h->d_stop_at, std::vector<long long>(n, -1)));
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
    TRY(dalloc(h, &h->d_cand_late, cap));
    TRY(dalloc(h, (char**)&h->d_cands,
               cap * (h->precision == 64 ? sizeof(Cand<double>) : sizeof(Cand<float>))));
    TRY(upload(h, &h->d_gap_head, std::vector<unsigned long long>(cap + NL + 1, 0ull)));
    TRY(upload(h, &h->d_head, std::vector<unsigned long long>(NL, 0ull)));
    TRY(upload(h, &h->d_enter, std::vector<int32_t>(NL, 0)));
    TRY(upload(h, &h->d_leave, std::vector<int32_t>(NL, 0)));
    h->n_lane_tiles = lane_tiles(h, 2);  // look-back words for the smaller tile
    h->max_slot_tiles = (NV + TILE - 1) / TILE + 1;
    h->n_junc_chunks = (NJ + JUNC_CHUNK - 1) / JUNC_CHUNK;
    TRY(upload(h, &h->d_lane_tiles, std::vector<unsigned long long>(h->n_lane_tiles, 0ull)));
    std::vector<Counters> c0(2, Counters{});
    c0[0].tag = 1;
    TRY(upload(h, &h->d_cnt, c0));
    TRY(upload(h, &h->d_bar, std::vector<unsigned>(2, 0u)));
    TRY(dalloc(h, &h->d_stage, 2 * std::max(NJ, 1)));
    CK(cudaHostAlloc((void**)&h->h_stage, sizeof(int32_t) * 2 * std::max(NJ, 1), cudaHostAllocDefault));
    CK(cudaHostAlloc((void**)&h->h_rb, sizeof(long long) * RB_WORDS * (MOSS_METRIC_SLOTS + 1),
                     cudaHostAllocDefault));
    for (int k = 0; k < MOSS_METRIC_SLOTS; ++k)
        CK(cudaEventCreateWithFlags(&h->rb_ev[k], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->stage_free, cudaEventDisableTiming));
    CK(cudaEventRecord(h->stage_free, h->stream));
    CK(cudaEventCreateWithFlags(&h->load_free, cudaEventDisableTiming));
    CK(cudaEventRecord(h->load_free, h->stream));
    for (int k = 0; k <= N_STEP_KERNELS; ++k) CK(cudaEventCreate(&h->ev[k]));
    TRY(junction_init(h, 0, NJ));
    CK(cudaStreamSynchronize(h->stream));
    TRY(build_graphs(h));
    return MOSS_OK;
}

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
    h->junc_offset.assign(NJ, 0); h->phase_green.assign(tot_ph, 0); h->phase_amber.assign(tot_ph, 0);
    h->route_span.resize(NV); h->routes.resize(tot_routes); h->dep.resize(NV);
    h->start_lane.resize(NV); h->v0f.resize(NV); h->veh_scen.resize(NV);
    h->scen_veh_off.assign(n + 1, 0); h->scen_lane_off.assign(n + 1, 0); h->scen_junc_off.assign(n + 1, 0);
    h->scen_road_off.assign(n + 1, 0);
    h->scen_lanes.assign(n, make_int4(0, 0, 0, 0));
    h->scen_nv.assign(n, 0); h->scen_nl.assign(n, 0); h->scen_nj.assign(n, 0); h->scen_nr.assign(n, 0);
    h->jl_plans.assign(tot_lanes, 0xff);
    h->road_span.assign(tot_roads, make_int2(0, 0));
    h->key0.resize(n); h->key1.resize(n);
    int LO = 0, JO = 0, VO = 0, RO = 0, PO = 0, ROFF = 0;
    for (int k = 0; k < n; ++k) {
        const MossNetwork& nt = nets[k];
        const MossVehicles& vh = vehs[k];
        fill_scenario(h, k, nt, vh, prms[k], LO, JO, VO, RO, PO, ROFF);
        const int nph = nt.n_junctions ? nt.junc_phase_off[nt.n_junctions] : 0;
        ROFF += vh.n ? vh.route_off[vh.n] : 0;
        h->scen_nv[k] = vh.n; h->scen_nl[k] = nt.n_lanes; h->scen_nj[k] = nt.n_junctions; h->scen_nr[k] = nt.n_roads;
        LO += nt.n_lanes; JO += nt.n_junctions; VO += vh.n; RO += nt.n_roads; PO += nph;
        h->scen_veh_off[k + 1] = VO; h->scen_lane_off[k + 1] = LO; h->scen_junc_off[k + 1] = JO;
        h->scen_road_off[k + 1] = RO;
    }
    h->junc_phase_off[NJ] = PO;
    // departure queues per start lane ordered by (dep, id) (R18)
    h->q_off.assign(NL + 1, 0);
    h->q_head.assign(std::max(NL, 1), 0);
    h->q_ids.resize(NV);
    build_queues(h, 0, NL, 0, NV, 0, NV);
    h->q_head.resize(NL);
    h->start_lanes.clear();
    for (int l = 0; l < NL; ++l)
        if (h->q_off[l + 1] > h->q_off[l]) h->start_lanes.push_back(l);
    if (!h->lane_groups) h->lane_groups = has_lane_groups(h, 0, (int)tot_roads);
    // junction lanes grouped by junction
    int n_jl = 0;
    for (int l = 0; l < NL; ++l) n_jl += h->lanes[l].lo < 0;
    h->jj_off.assign(NJ + 1, 0);
    h->jj_lane.assign(n_jl, 0); h->jj_from.assign(n_jl, 0);
    build_jj(h, 0, NJ, 0, NL, 0, n_jl, 0);
    return device_setup(h, stream);
}

// ---- slot batches (serving): scenarios loaded into fixed-capacity slots ----

// lanes [l0, l1) of slot k as padding: isolated one-lane roads of 1 m (road
// rpad) with no junction lanes and no vehicles
void fill_padding(MossHandle* h, int k, int l0, int l1, int rpad) {
    for (int l = l0; l < l1; ++l) {
        LaneInfo& li = h->lanes[l];
        li.L = 1.0f; li.vmax = 1.0f;
        li.lo = l; li.hi = l + 1; li.jb = l0; li.je = l0;
        li.road = rpad; li.scen = (unsigned short)k; li.flags = 0;
        h->lane_src_road[l] = -1;
        h->jl_plans[l] = 0xff;
    }
}

// slot k empty: every lane, road and junction padding, no vehicles (with
// vehicles: also every vehicle and route entry of its capacity, else only the
// ones the slot's last scenario used)
void clear_slot(MossHandle* h, int k, bool vehicles) {
    const SlotInfo& S = h->slot[k];
    const int lpad = S.LO + S.nl_cap - 1, rpad = S.RO + S.nr_cap - 1;
    fill_padding(h, k, S.LO, S.LO + S.nl_cap, rpad);
    for (int r = S.RO; r < S.RO + S.nr_cap; ++r) h->road_span[r] = make_int2(lpad, lpad + 1);
    for (int j = S.JO; j < S.JO + S.nj_cap; ++j) {
        h->junc_scen[j] = k; h->junc_offset[j] = 0; h->junc_phase_off[j] = S.PO;
    }
    h->junc_phase_off[S.JO + S.nj_cap] = S.PO + S.np_cap;  // the padding junction owns the spare phases
    for (int q = S.PO; q < S.PO + S.np_cap; ++q) { h->phase_green[q] = 1; h->phase_amber[q] = 0; }
    const int nv = vehicles ? S.nv_cap : h->scen_nv[k];
    for (int g = S.VO; g < S.VO + nv; ++g) {
        h->route_span[g] = make_int2(S.QO, S.QO);
        h->dep[g] = 0; h->start_lane[g] = lpad; h->v0f[g] = 1.0f; h->veh_scen[g] = k;
    }
    if (vehicles)
        for (int q = S.QO; q < S.QO + S.nq_cap; ++q) h->routes[q] = rpad;
    build_queues(h, S.LO, S.LO + S.nl_cap, S.VO, S.VO, S.VO, S.VO + S.nv_cap);
    for (int q = 0; q < S.nl_cap; ++q) h->start_lanes[S.SO + q] = lpad;
    build_jj(h, S.JO, S.JO + S.nj_cap, S.LO, S.LO + S.nl_cap, S.JJ, S.JJ + S.njj_cap, lpad);
    h->scen_nv[k] = 0; h->scen_nl[k] = 0; h->scen_nj[k] = 0; h->scen_nr[k] = 0;
}

int create_slots_impl(int n, const MossSlotCaps* caps, const MossParams* prm, void* stream, MossHandle* h) {
    if (n < 1 || n > 65535) return fail(h, MOSS_EINVAL, "1 to 65535 slots");
    if (!caps || !prm) return fail(h, MOSS_EINVAL, "null argument");
    if (prm->delta != 4.0) return fail(h, MOSS_EINVAL, "only delta = 4 is supported");
    if (prm->precision != 32 && prm->precision != 64) return fail(h, MOSS_EINVAL, "precision must be 32 or 64");
    h->prm = *prm;
    h->precision = prm->precision;
    h->n_scen = n;
    h->slots = true;
    h->slot.resize(n);
    long long L = 0, R = 0, J = 0, P = 0, JJ = 0, V = 0, Q = 0, S = 0;
    for (int k = 0; k < n; ++k) {
        const MossSlotCaps& c = caps[k];
        if (c.n_lanes < 0 || c.n_roads < 0 || c.n_junctions < 0 || c.n_phases < 0 || c.n_vehicles < 0 ||
            c.n_route_entries < 0)
            return fail(h, MOSS_EINVAL, "negative slot capacity");
        SlotInfo& si = h->slot[k];
        // one padding lane, road and junction beyond the stated capacity
        si.LO = (int)L; si.nl_cap = c.n_lanes + 1;
        si.RO = (int)R; si.nr_cap = c.n_roads + 1;
        si.JO = (int)J; si.nj_cap = c.n_junctions + 1;
        si.PO = (int)P; si.np_cap = c.n_phases;
        si.JJ = (int)JJ; si.njj_cap = c.n_lanes;
        si.VO = (int)V; si.nv_cap = c.n_vehicles;
        si.QO = (int)Q; si.nq_cap = c.n_route_entries;
        si.SO = (int)S;
        L += si.nl_cap; R += si.nr_cap; J += si.nj_cap; P += si.np_cap; JJ += si.njj_cap; V += si.nv_cap;
        Q += si.nq_cap; S += si.nl_cap;
    }
    if (L >= (1ll << 30) || V >= (1ll << 30) || Q >= (1ll << 31) - 1 || R >= (1ll << 30) || JJ >= (1ll << 30))
        return fail(h, MOSS_EINVAL, "slot capacities too large for 32-bit indices");
    h->n_lanes = (int)L; h->n_junctions = (int)J; h->n_veh = (int)V; h->n_phases = (int)P;
    h->lanes.assign(L, LaneInfo{});
    h->lane_src_road.assign(L, -1);
    h->junc_scen.assign(J, 0); h->junc_phase_off.assign(J + 1, 0);
    h->junc_offset.assign(J, 0); h->phase_green.assign(P, 1); h->phase_amber.assign(P, 0);
    h->route_span.assign(V, make_int2(0, 0)); h->routes.assign(Q, 0); h->dep.assign(V, 0);
    h->start_lane.assign(V, 0); h->v0f.assign(V, 1.0f); h->veh_scen.assign(V, 0);
    h->scen_veh_off.assign(n + 1, 0); h->scen_lane_off.assign(n + 1, 0); h->scen_junc_off.assign(n + 1, 0);
    h->scen_road_off.assign(n + 1, 0);
    h->scen_lanes.assign(n, make_int4(0, 0, 0, 0));
    h->scen_nv.assign(n, 0); h->scen_nl.assign(n, 0); h->scen_nj.assign(n, 0); h->scen_nr.assign(n, 0);
    h->jl_plans.assign(L, 0xff);
    h->road_span.assign(R, make_int2(0, 0));
    h->key0.assign(n, 0); h->key1.assign(n, 0);
    h->q_off.assign(L + 1, 0); h->q_head.assign(L, 0); h->q_ids.assign(std::max<long long>(V, 1), 0);
    h->start_lanes.assign(S, 0);
    h->jj_off.assign(J + 1, 0); h->jj_lane.assign(JJ, 0); h->jj_from.assign(JJ, 0);
    for (int k = 0; k < n; ++k) {
        const SlotInfo& si = h->slot[k];
        h->scen_veh_off[k + 1] = si.VO + si.nv_cap; h->scen_lane_off[k + 1] = si.LO + si.nl_cap;
        h->scen_junc_off[k + 1] = si.JO + si.nj_cap; h->scen_road_off[k + 1] = si.RO + si.nr_cap;
        clear_slot(h, k, true);
        h->key0[k] = (uint32_t)(prm->seed & 0xffffffffull);
        h->key1[k] = (uint32_t)(prm->seed >> 32) ^ (prm->scenario + (uint32_t)k);
    }
    h->q_ids.resize(V);
    h->lane_groups = false;
    return device_setup(h, stream);
}

// Asynchronous upload of host ranges through the pinned load staging area:
// the copies run in stream order behind the work already queued (so a slot's
// tables are replaced only after the steps enqueued before the load), and the
// host does not wait for them.
struct Stager {
    MossHandle* h;
    size_t off = 0;
    template <typename T>
    int put(T* d, const std::vector<T>& v, long long b, long long cnt) {
        return put_ptr(d + b, v.data() + b, cnt);
    }
    template <typename T>
    int put_ptr(T* d, const T* src, long long cnt) {
        if (cnt <= 0) return MOSS_OK;
        const size_t nb = (size_t)cnt * sizeof(T);
        std::memcpy(h->h_load + off, src, nb);
        CK(cudaMemcpyAsync(d, h->h_load + off, nb, cudaMemcpyHostToDevice, h->stream));
        off += (nb + 15) & ~size_t(15);
        return MOSS_OK;
    }
};

// room for `bytes` in the load staging area once the previous load's copies ran
int stage_reserve(MossHandle* h, size_t bytes) {
    CK(cudaEventSynchronize(h->load_free));
    if (bytes > h->load_cap) {
        if (h->h_load) cudaFreeHost(h->h_load);
        h->h_load = nullptr;
        h->load_cap = 0;
        CK(cudaHostAlloc((void**)&h->h_load, bytes, cudaHostAllocDefault));
        h->load_cap = bytes;
    }
    return MOSS_OK;
}

int load_slot_impl(MossHandle* h, int k, const MossNetwork* net, const MossVehicles* veh, const MossParams* prm) {
    if (!h->slots) return fail(h, MOSS_EINVAL, "not a slot batch (moss_slots_create)");
    if (k < 0 || k >= h->n_scen) return fail(h, MOSS_EINVAL, "slot index out of range");
    std::vector<std::vector<int32_t>> outs;
    TRY(validate(h, net, veh, prm, &outs));
    if (!same_model(h->prm, *prm)) return fail(h, MOSS_EINVAL, "the slot batch's model parameters differ");
    SlotInfo& S = h->slot[k];
    if (S.loaded && !S.retired) return fail(h, MOSS_EINVAL, "slot in use: retire it first");
    if (S.loaded && h->steps_enqueued <= S.retire_step)
        return fail(h, MOSS_EINVAL, "retired slot still holds its vehicles: step once first");
    const int nph = net->n_junctions ? net->junc_phase_off[net->n_junctions] : 0;
    const int nq = veh->n ? veh->route_off[veh->n] : 0;
    if (net->n_lanes > S.nl_cap - 1 || net->n_roads > S.nr_cap - 1 || net->n_junctions > S.nj_cap - 1 ||
        nph > S.np_cap || net->n_lanes - net->n_road_lanes > S.njj_cap || veh->n > S.nv_cap || nq > S.nq_cap)
        return fail(h, MOSS_EINVAL, "scenario larger than the slot's capacity");
    clear_slot(h, k, false);
    fill_scenario(h, k, *net, *veh, *prm, S.LO, S.JO, S.VO, S.RO, S.PO, S.QO);
    if (has_lane_groups(h, S.RO, S.RO + net->n_roads) || net->jl_plans) {
        h->lane_groups = false;
        clear_slot(h, k, false);
        return fail(h, MOSS_EINVAL, "slot batches take networks without lane groups or plans");
    }
    // padding junction after the scenario's junctions owns the spare phases
    for (int j = S.JO + net->n_junctions; j <= S.JO + S.nj_cap; ++j) h->junc_phase_off[j] = S.PO + nph;
    h->junc_phase_off[S.JO + S.nj_cap] = S.PO + S.np_cap;
    build_queues(h, S.LO, S.LO + S.nl_cap, S.VO, S.VO + veh->n, S.VO, S.VO + S.nv_cap);
    {
        int q = S.SO;
        for (int l = S.LO; l < S.LO + S.nl_cap; ++l)
            if (h->q_off[l + 1] > h->q_off[l] && l < S.LO + net->n_lanes) h->start_lanes[q++] = l;
        for (; q < S.SO + S.nl_cap; ++q) h->start_lanes[q] = S.LO + S.nl_cap - 1;
    }
    build_jj(h, S.JO, S.JO + S.nj_cap, S.LO, S.LO + S.nl_cap, S.JJ, S.JJ + S.njj_cap, S.LO + S.nl_cap - 1);
    // device ranges of the slot (asynchronous, in stream order)
    std::vector<JuncInfo> junc(S.nj_cap);
    for (int q = 0; q < S.nj_cap; ++q) {
        const int j = S.JO + q;
        junc[q].offset = h->junc_offset[j];
        junc[q].phase_off = h->junc_phase_off[j];
        junc[q].np = q + 1 < S.nj_cap ? h->junc_phase_off[j + 1] - h->junc_phase_off[j] : 0;
        junc[q].scen = k;
    }
    const std::vector<int4> mp0(S.nj_cap, make_int4(0, 1, -1, 0));
    const size_t need = 16 * 26 + sizeof(LaneInfo) * S.nl_cap + sizeof(JuncInfo) * S.nj_cap + 8 * (size_t)S.np_cap +
                        sizeof(int4) * S.nj_cap + 4 * (size_t)(S.nj_cap + 1) + 8 * (size_t)S.njj_cap +
                        sizeof(int2) * S.nr_cap + 4 * (size_t)S.nl_cap + sizeof(int2) * (size_t)S.nv_cap +
                        4 * (size_t)S.nq_cap + 12 * (size_t)S.nv_cap + 4 * (size_t)(S.nl_cap + 1) +
                        8 * (size_t)S.nl_cap + 16 + sizeof(int4);
    TRY(stage_reserve(h, need));
    Stager st{h};
    TRY(st.put(h->d_lane, h->lanes, S.LO, S.nl_cap));
    TRY(st.put_ptr(h->d_junc + S.JO, junc.data(), S.nj_cap));
    TRY(st.put(h->d_phase_green, h->phase_green, S.PO, S.np_cap));
    TRY(st.put(h->d_phase_amber, h->phase_amber, S.PO, S.np_cap));
    TRY(st.put_ptr(h->d_mp + S.JO, mp0.data(), S.nj_cap));
    TRY(st.put(h->d_jj_off, h->jj_off, S.JO, S.nj_cap + 1));
    TRY(st.put(h->d_jj_lane, h->jj_lane, S.JJ, S.njj_cap));
    TRY(st.put(h->d_jj_from, h->jj_from, S.JJ, S.njj_cap));
    TRY(st.put(h->d_road_span, h->road_span, S.RO, S.nr_cap));
    TRY(st.put(h->d_jl_plans, h->jl_plans, S.LO, S.nl_cap));
    // vehicles and route entries past the scenario's are never read (they
    // are in no queue): only the used parts go up
    TRY(st.put(h->d_route_span, h->route_span, S.VO, veh->n));
    TRY(st.put(h->d_routes, h->routes, S.QO, nq));
    TRY(st.put(h->d_dep, h->dep, S.VO, veh->n));
    TRY(st.put(h->d_v0f, h->v0f, S.VO, veh->n));
    TRY(st.put(h->d_q_off, h->q_off, S.LO, S.nl_cap + 1));
    TRY(st.put(h->d_q_ids, h->q_ids, S.VO, veh->n));
    TRY(st.put(h->d_q_head, h->q_head, S.LO, S.nl_cap));
    TRY(st.put(h->d_start_lanes, h->start_lanes, S.SO, S.nl_cap));
    TRY(st.put(h->d_key0, h->key0, k, 1));
    TRY(st.put(h->d_key1, h->key1, k, 1));
    TRY(st.put(h->d_scen_lanes, h->scen_lanes, k, 1));
    CK(cudaEventRecord(h->load_free, h->stream));
    // fixed-time policy (0), no manual phase, no pressure, every vehicle
    // waiting (0) without flags, clock and metrics at 0, running (control 0),
    // no horizon (-1)
    CK(cudaMemsetAsync(h->d_junc_policy + S.JO, 0, 4 * (size_t)S.nj_cap, h->stream));
    CK(cudaMemsetAsync(h->d_junc_manual + S.JO, 0, 4 * (size_t)S.nj_cap, h->stream));
    CK(cudaMemsetAsync(h->d_mp_press + (size_t)S.JO * 8, 0, 32 * (size_t)S.nj_cap, h->stream));
    if (veh->n > 0) {
        CK(cudaMemsetAsync(h->d_vstatus + S.VO, 0, 4 * (size_t)veh->n, h->stream));
        CK(cudaMemsetAsync(h->d_vflags + S.VO, 0, 4 * (size_t)veh->n, h->stream));
    }
    CK(cudaMemsetAsync(h->d_step + k, 0, 8, h->stream));
    CK(cudaMemsetAsync(h->d_metrics + (size_t)k * M_NFIELDS, 0, 8 * (size_t)M_NFIELDS, h->stream));
    CK(cudaMemsetAsync(h->d_scen_ctl + k, 0, 4, h->stream));
    CK(cudaMemsetAsync(h->d_stop_at + k, 0xff, 8, h->stream));
    TRY(junction_init(h, S.JO, S.JO + S.nj_cap));
    h->scen_nv[k] = veh->n; h->scen_nl[k] = net->n_lanes; h->scen_nj[k] = net->n_junctions;
    h->scen_nr[k] = net->n_roads;
    S.loaded = true;
    S.retired = false;
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
    if (h->load_free) cudaEventDestroy(h->load_free);
    if (h->h_load) cudaFreeHost(h->h_load);
    h->h_load = nullptr;
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
    const int nv = h->scen_nv[s];
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
    const int v0 = h->scen_veh_off[s], v1 = v0 + h->scen_nv[s];
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
    if (h->slots) return fail(h, MOSS_EINVAL, "lane setters are not available on slot batches");
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
    if (h->slots) return fail(h, MOSS_EINVAL, "re-routing is not available on slot batches");
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
        const int l0 = h->scen_lane_off[s], l1 = l0 + h->scen_nl[s];
        if (l1 > l0) {
            k_lane_queue<Real><<<(l1 - l0 + 255) / 256, 256, 0, h->stream>>>(c, l0, l1, (int32_t*)h->d_mbuf);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(queue, h->d_mbuf, (size_t)(l1 - l0) * 4, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
    }
    if (speed) {
        const int r0 = h->scen_road_off[s], r1 = r0 + h->scen_nr[s];
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
    h->steps_enqueued += n;
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
    const int j0 = h->scen_junc_off[scenario], nj = h->scen_nj[scenario];
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

int moss_batch_set_signal_phases(moss_t h, int n, const int32_t* scenarios, const int32_t* junction_ids,
                                 const int32_t* phase_idx) {
    if (!h) return MOSS_EINVAL;
    if (n < 0 || (n > 0 && (!scenarios || !junction_ids || !phase_idx))) return fail(h, MOSS_EINVAL, "bad arrays");
    if (n > h->n_junctions) return fail(h, MOSS_EINVAL, "more entries than the batch has junctions");
    if (n == 0) return MOSS_OK;
    CK(cudaEventSynchronize(h->stage_free));
    int32_t* sj = h->h_stage;
    int32_t* sp = h->h_stage + n;
    for (int k = 0; k < n; ++k) {
        const int s = scenarios[k], j = junction_ids[k], p = phase_idx[k];
        if (s < 0 || s >= h->n_scen) return fail(h, MOSS_EINVAL, "scenario out of range");
        if (j < 0 || j >= h->scen_nj[s]) return fail(h, MOSS_EINVAL, "junction id out of range");
        const int g = h->scen_junc_off[s] + j;
        const int np = h->junc_phase_off[g + 1] - h->junc_phase_off[g];
        if (p < 0 || p >= std::max(np, 1)) return fail(h, MOSS_EINVAL, "phase index out of range");
        sj[k] = g;
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
    if (h->slots) return fail(h, MOSS_EINVAL, "signal policies are not available on slot batches");
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
    if (h->slots) return fail(h, MOSS_EINVAL, "lane plans are not available on slot batches");
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
    if (h->n_scen != 1 || h->slots) return fail(h, MOSS_EINVAL, "moss_set_state takes single-scenario handles");
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
    c.n_cur = (int)n_act; c.n_ent = 0; c.n_cand = 0; c.n_late = 0; c.ticket_lane = 0; c.res_done = 0;
    CK(cudaMemcpy(h->d_cnt + h->parity, &c, sizeof(c), cudaMemcpyHostToDevice));
    TRY(junction_init(h, 0, h->n_junctions));
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

int moss_slots_create(int n, const MossSlotCaps* caps, const MossParams* prm, void* cuda_stream,
                      const MossAllocator* allocator, moss_t* out) {
    if (!out) return MOSS_EINVAL;
    *out = nullptr;
    if (allocator && (!allocator->alloc || !allocator->release)) return MOSS_EINVAL;
    MossHandle* h = new (std::nothrow) MossHandle();
    if (!h) return MOSS_ENOMEM;
    if (allocator) h->allocator = *allocator;
    int rc;
    try {
        rc = create_slots_impl(n, caps, prm, cuda_stream, h);
    } catch (const std::bad_alloc&) {
        rc = fail(h, MOSS_ENOMEM, "host allocation failed");
    }
    if (rc != MOSS_OK) {
        fprintf(stderr, "moss_slots_create: %s\n", h->err.c_str());
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return MOSS_OK;
}

int moss_slot_load(moss_t h, int slot, const MossNetwork* net, const MossVehicles* veh, const MossParams* prm) {
    if (!h) return MOSS_EINVAL;
    if (!net || !veh || !prm) return fail(h, MOSS_EINVAL, "null argument");
    try {
        return load_slot_impl(h, slot, net, veh, prm);
    } catch (const std::bad_alloc&) {
        return fail(h, MOSS_ENOMEM, "host allocation failed");
    }
}

int moss_slot_retire(moss_t h, int slot) {
    if (!h) return MOSS_EINVAL;
    if (!h->slots) return fail(h, MOSS_EINVAL, "not a slot batch");
    if (slot < 0 || slot >= h->n_scen) return fail(h, MOSS_EINVAL, "slot index out of range");
    SlotInfo& S = h->slot[slot];
    if (!S.loaded || S.retired) return MOSS_OK;
    k_put_i32<<<1, 1, 0, h->stream>>>(h->d_scen_ctl + slot, SC_RETIRE | SC_FROZEN);
    CK(cudaGetLastError());
    S.retired = true;
    S.retire_step = h->steps_enqueued;
    h->scen_nv[slot] = 0; h->scen_nl[slot] = 0; h->scen_nj[slot] = 0; h->scen_nr[slot] = 0;
    return MOSS_OK;
}

int moss_slot_set_horizon(moss_t h, int slot, int64_t stop_at) {
    if (!h) return MOSS_EINVAL;
    if (!h->slots) return fail(h, MOSS_EINVAL, "not a slot batch");
    if (slot < 0 || slot >= h->n_scen) return fail(h, MOSS_EINVAL, "slot index out of range");
    if (!h->slot[slot].loaded || h->slot[slot].retired) return fail(h, MOSS_EINVAL, "slot not loaded");
    k_put_i64<<<1, 1, 0, h->stream>>>(h->d_stop_at + slot, stop_at < 0 ? -1ll : (long long)stop_at);
    CK(cudaGetLastError());
    return MOSS_OK;
}

int moss_set_step_mode(moss_t h, int mode) {
    if (!h) return MOSS_EINVAL;
    if (mode != 0 && mode != 1) return fail(h, MOSS_EINVAL, "step mode must be 0 or 1");
    if (mode == 1) {
        int coop = 0;
        CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
        if (!coop) return fail(h, MOSS_EINVAL, "the device has no cooperative launch");
    }
    CK(cudaStreamSynchronize(h->stream));
    const int old = h->step_mode;
    h->step_mode = mode;
    destroy_graphs(h);
    const int rc = build_graphs(h);
    if (rc != MOSS_OK) {
        h->step_mode = old;
        destroy_graphs(h);
        TRY(build_graphs(h));
        return rc;
    }
    return MOSS_OK;
}

int moss_step_launches(moss_t h, int* out) {
    if (!h || !out) return MOSS_EINVAL;
    *out = h->step_mode == 1 ? 1 : (MOSS_FOLD_RESOLVE ? 3 : 4);
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
    // coordinate search over the schedule: blocks per SM of each kernel, the
    // road-lane weight of k_decide's runs, the lane-scan tile and the step
    // mode; results do not depend on the schedule, only the time does
    int coop = 0;
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
    struct Knob { int* v; int n; int c[3]; };
    const Knob knobs[] = {
        {&h->cfg_decide, 3, {3, 4, 5}},   {&h->cfg_runw, 3, {0, 1, 2}}, {&h->cfg_lanescan, 3, {1, 2, 4}},
        {&h->cfg_lsr, 2, {4, 2, 0}},      {&h->cfg_place, 3, {4, 8, 16}}, {&h->step_mode, coop ? 2 : 1, {0, 1, 0}},
    };
    for (const Knob& kb : knobs) {
        int best = *kb.v;
        double best_ms = 1e300;
        for (int k = 0; k < kb.n; ++k) {
            *kb.v = kb.c[k];
            h->launch_err = cudaSuccess;
            double ms = 0;
            TRY(time_steps(h, trial_steps, &ms));
            if (h->launch_err != cudaSuccess) {  // a mode this device cannot launch
                h->launch_err = cudaSuccess;
                continue;
            }
            if (ms < best_ms) { best_ms = ms; best = kb.c[k]; }
        }
        *kb.v = best;
    }
    destroy_graphs(h);
    TRY(build_graphs(h));
    if (chosen3) { chosen3[0] = h->cfg_decide; chosen3[1] = h->cfg_lanescan; chosen3[2] = h->cfg_place; }
    return check_device(h);
}

int moss_get_schedule(moss_t h, int* out7) {
    if (!h || !out7) return MOSS_EINVAL;
    out7[0] = h->cfg_decide; out7[1] = h->cfg_lanescan; out7[2] = h->cfg_place;
    out7[3] = h->cfg_runw; out7[4] = 4 * h->cfg_lsr; out7[5] = h->step_mode; out7[6] = h->cfg_ccap;
    return MOSS_OK;
}

int moss_set_schedule(moss_t h, const int* in7) {
    if (!h || !in7) return MOSS_EINVAL;
    const int* in6 = in7;
    if (in6[0] < 1 || in6[0] > 16 || in6[1] < 1 || in6[1] > 32 || in6[2] < 1 || in6[2] > 32 || in6[3] < 0 ||
        in6[3] > 8 || (in6[4] != 8 && in6[4] != 16) || (in6[5] != 0 && in6[5] != 1) || in7[6] < 0 ||
        in7[6] > CAND_LOCAL)
        return fail(h, MOSS_EINVAL, "schedule value out of range");
    if (in6[5] == 1) {
        int coop = 0;
        CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
        if (!coop) return fail(h, MOSS_EINVAL, "the device has no cooperative launch");
    }
    CK(cudaStreamSynchronize(h->stream));
    const int old[7] = {h->cfg_decide, h->cfg_lanescan, h->cfg_place, h->cfg_runw, h->cfg_lsr, h->step_mode,
                        h->cfg_ccap};
    h->cfg_decide = in6[0]; h->cfg_lanescan = in6[1]; h->cfg_place = in6[2];
    h->cfg_runw = in6[3]; h->cfg_lsr = in6[4] / 4; h->step_mode = in6[5]; h->cfg_ccap = in7[6];
    destroy_graphs(h);
    const int rc = build_graphs(h);
    if (rc != MOSS_OK) {
        h->cfg_decide = old[0]; h->cfg_lanescan = old[1]; h->cfg_place = old[2];
        h->cfg_runw = old[3]; h->cfg_lsr = old[4]; h->step_mode = old[5]; h->cfg_ccap = old[6];
        destroy_graphs(h);
        TRY(build_graphs(h));
        return rc;
    }
    return MOSS_OK;
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
