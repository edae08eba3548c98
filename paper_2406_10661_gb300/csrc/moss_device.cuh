// Device side of the per-timestep vehicle update (arxiv 2406.10661, §3.1,
// App. B.2-B.3), written for sm_103a.
//
// Layout.  Active vehicles live in a lane-major snapshot sorted by (lane,
// s descending, id ascending); lane l occupies slots [off[l], off[l+1]).
// Each slot holds two 16-byte records: A = (s, v, id, lane) and B = (v0f,
// route index of the current road, route index of the last road, next lane).
// The snapshot of step t is read-only during step t (§3.1 two-phase
// read/write separation); step t writes the snapshot of step t+1 into the
// other buffer.  The paper's linked lists with side pointers (§3.1) become
// O(1) neighbour slots (leader = slot-1, follower = slot+1) and a binary
// search in the adjacent lane's segment (adjacent lanes of a road are
// adjacent in memory).
//
// One step = three kernels:
//   k_decide    per vehicle: sensing, IDM (App. B.3 eqs. (1)-(2)), the
//               randomized MOBIL decision (App. B.3; run from a per-warp
//               shared-memory queue of the vehicles whose attempt draw
//               passed), ballistic integration with clamps, transfer at lane
//               ends and arrival (App. B.2 update stream 1); each block
//               takes a run of whole roads and at its end resolves the
//               lane-change candidates of its run (deterministic conflict
//               rule between candidates entering the same gap from both
//               sides); extra blocks run the departure insertion (App. B.2
//               update stream 3);
//   k_lanescan  first tickets: the fit of the next step's run weight, the
//               candidates past a decide block's own list, max-pressure
//               phase sums (§3.2); then per-lane sizes of the next snapshot
//               -> offsets (single-pass decoupled look-back scan), signal
//               states of the next step (§3.2 policies);
//   k_place     writes the next snapshot: vehicles that kept their lane keep
//               their relative order (no overtaking within a lane), vehicles
//               that entered a lane are merged by (s, id).
// (k_step_coop runs the same three as phases of one cooperative launch.)
#pragma once

#include <cuda/atomic>
#include <stdint.h>

namespace moss {

enum : int { LIGHT_GREEN = 0, LIGHT_AMBER = 1, LIGHT_RED = 2 };
enum : int { POL_FIXED = 0, POL_MANUAL = 1, POL_NONE = 2, POL_MAXP = 3 };
enum : int {
    F_FLAGGED = 1, F_CHANGED = 2, F_CANDIDATE = 4, F_TRANSFER = 8,
    F_ARRIVED = 16, F_INSERTED = 32, F_CONFLICT_LOST = 64
};
enum : int8_t { C_STAY = 0, C_MOVE = 1, C_ARRIVE = 2 };

// per-scenario metric accumulators (int64, deterministic integer sums)
enum : int {
    M_UPDATES = 0, M_ARRIVED, M_TT_STEPS, M_SPEED_FX, M_LANE_CHANGES, M_FLAGGED,
    M_OVERLAPS, M_INSERTED, M_ERRORS, M_CUR_ACTIVE, M_CUR_ARRIVED, M_MOBIL, M_NFIELDS
};
constexpr double SPEED_FX = 16777216.0;  // speed sums in units of 2^-24 m/s

// per-scenario control (slot batches): a frozen scenario does not advance
// (its vehicles keep their state, its clock and signals stand still); a
// retiring one has its vehicles removed by the next step
enum : int { SC_FROZEN = 1, SC_RETIRE = 2 };

// device error bits (Counters::err)
enum : int { ERR_TIMEOUT = 1, ERR_ROUTE = 2, ERR_TRANSFER = 4, ERR_RANGE = 8 };
// errors after which the state can no longer be trusted: every later kernel
// of the handle returns at once and the host reports the error
constexpr int ERR_POISON = ERR_TIMEOUT | ERR_RANGE;

constexpr int TILE = 256;           // slots per tile of k_decide / k_place (= threads)
constexpr int LANESCAN_THREADS = 256;
constexpr int LANESCAN_ITEMS = 16;
constexpr int LANESCAN_TILE = LANESCAN_THREADS * LANESCAN_ITEMS;
constexpr int JUNC_CHUNK = 256;     // junctions per k_lanescan ticket (one per thread)
constexpr int RUNSTAT_MAX = 4096;  // k_decide work blocks whose run statistics are kept
constexpr long long SPIN_LIMIT = 1ll << 22;  // bounded waits (~0.5 s with backoff)

// Step counters, one set per parity of the ping-pong snapshots: step t uses
// the set of its parity and prepares the other one for step t + 1 (that set
// was last used by step t - 1, which has finished).  err lives in set 0.
struct Counters {
    int n_cur;       // active vehicles in the current snapshot
    int n_ent;       // entrants appended this step
    int n_cand;      // lane-change candidates listed this step (for k_resolve)
    int ticket_lane; // k_lanescan tickets
    int n_late;      // candidates left to k_lanescan (past a k_decide block's own list)
    int tag;         // step tag of the per-lane lists (never 0)
    int err;         // device error bits (set 0 only)
    int n_mp;        // junctions under max pressure (set 0 only)
    int res_done;    // k_lanescan tickets of candidate / pressure work finished
    int run_wq;      // fitted weight of a road-lane slot in k_decide's runs, x256 (0: none yet)
    int n_runs;      // k_decide work runs of this step (their statistics for the fit)
};

// the candidates past a decide block's own list are resolved in the first
// tickets of k_lanescan instead of a kernel of their own
#ifndef MOSS_FOLD_RESOLVE
#define MOSS_FOLD_RESOLVE 1
#endif

// snapshot records
template <typename Real> struct RecA;
template <> struct alignas(16) RecA<float> { float s, v; int id, lane; };
template <> struct alignas(16) RecA<double> { double s, v; int id, lane; };
// a record that belongs to no lane (neighbour slot outside the snapshot)
template <typename Real> __host__ __device__ __forceinline__ RecA<Real> no_rec() {
    RecA<Real> r;
    r.s = Real(0); r.v = Real(0); r.id = -1; r.lane = -1;
    return r;
}
struct alignas(16) RecB {
    float v0f;
    int rptr;   // index in routes[] of the current road (junction lane: the road just left)
    int rlast;  // index in routes[] of the last road
    int nl;     // next lane on the route (-1 on the last road)
};
template <typename Real> struct alignas(2 * sizeof(Real)) SV { Real s, v; };

// A lane-change candidate, finished by k_resolve.  gap = its insertion
// position in the target lane's segment plus the target lane's index: equal
// for two candidates exactly when they enter the same lane between the same
// target leader and follower (unique over lanes: lane l's positions span
// [off[l], off[l+1]], shifted by l).  Candidates of one gap form a list
// (gap_head, next).  The record carries everything the update needs for
// either outcome: the vehicle's records and its kinematics on the target
// lane (granted) and on its own lane (lost a conflict).
template <typename Real>
struct alignas(16) Cand {
    RecA<Real> E;            // the vehicle's snapshot records
    RecB EB;
    int slot, gap, next, bits;  // slot; gap key; list link; CB_* bits
    int nl, tnl, scen, pad;     // next lane from the own / the target lane; scenario
    Real u, scale;              // utility of the chosen side and its flag scale (R22)
    Real a, lgap, sgap;         // own lane: acceleration, leader gap, stop-line gap
    Real ta, tlgap, tsgap;      // target lane: the same
};
enum : int {
    CB_RIGHT = 1, CB_FLAG = 2, CB_LEADER = 4, CB_STOP = 8, CB_OVERLAP = 16, CB_TLEADER = 32, CB_TSTOP = 64,
    CB_TOVERLAP = 128
};

// One 32-byte record per lane.
//   road lane:     lo, hi = lanes [lo, hi) of its road (left to right); jb, je =
//                  junction lanes leaving it; road = its road; scen = scenario
//   junction lane: lo = -1, hi = the road lane it feeds; jb = its junction;
//                  je = phase mask; road = road of its target
//   flags: LF_* bits set by the lane setters
struct alignas(32) LaneInfo {
    float L, vmax;
    int lo, hi, jb, je, road;
    unsigned short scen, flags;
};
enum : int {
    LF_RESTRICTED = 1,  // restricted from passing: not entered (R25)
    LF_OFF = 2          // junction lane outside the current lane plan of its road (R28)
};

// One 16-byte record per junction (signal program; policy and manual phase
// are mutable and kept apart)
struct alignas(16) JuncInfo {
    int offset;    // program shift in steps
    int phase_off; // first phase in phase_green / phase_amber
    int np;        // number of phases (0 = no signal)
    int scen;      // scenario
};

template <typename Real>
struct Snap {
    RecA<Real>* a;
    RecB* b;
    int32_t* off;  // [n_lanes+1] lane segments
};

template <typename Real>
struct Ctx {
    // ---- network (possibly a union of scenarios)
    int n_lanes, n_junctions, n_scen, n_veh;
    const LaneInfo* lane;
    const JuncInfo* junc;
    const int32_t* phase_green;
    const int32_t* phase_amber;
    int32_t* junc_policy;
    int32_t* junc_manual;
    int32_t* junc_state;  // bits 0-3 phase, 4-7 n_phases, 8 amber, 9 all green, 10-13 phase after the amber
    int4* mp;             // max-pressure state per junction: phase, steps in the interval, phase after the amber (-1)
    const int32_t* jj_off;   // [n_junctions+1] junction lanes of each junction (CSR)
    const int32_t* jj_lane;  // absolute lane ids
    const int32_t* jj_from;  // the road lane each of them leaves
    const int2* road_span;   // [n_roads] (first, end) road lanes of every road (absolute ids)
    int n_jj;                // junction lanes in jj_lane
    int32_t* mp_press;       // [n_junctions][8] phase pressures of this step, summed by k_resolve
    int* n_mp;               // junctions under max pressure
    // ---- vehicles (by global id)
    const int2* route_span;  // [n_veh] route of a vehicle: routes[x .. y)
    const int32_t* routes;
    const int32_t* dep;
    const float* v0f;
    int32_t* vstatus;
    int32_t* vflags;  // (step & 0xFFFFFF) << 8 | flags, written when flags != 0
    // ---- departure queues (by lane) and the lanes that have one
    const int32_t* q_off;
    const int32_t* q_ids;
    int32_t* q_head;
    const int32_t* start_lanes;
    int n_start;
    // ---- scenarios
    const uint32_t* key0;
    const uint32_t* key1;
    const int32_t* veh_base;  // first global vehicle id of the scenario
    const int4* scen_lanes;   // first lane, first junction lane, end of the lanes in use
    long long* scen_step;
    long long* metrics;  // [n_scen][M_NFIELDS]
    int32_t* scen_ctl;   // [n_scen] SC_* bits (slot batches; 0 otherwise)
    const long long* stop_at;  // [n_scen] step at which a scenario freezes (-1: never)
    // ---- snapshots (current -> next)
    Snap<Real> cur, nxt;
    // ---- per-step scratch
    int8_t* code;         // per current slot: C_STAY / C_MOVE / C_ARRIVE
    SV<Real>* stay;       // stayer's new (s, v)
    RecA<Real>* ea;       // entrants of the next snapshot (lane changes, transfers, insertions)
    RecB* eb;
    int32_t* enext;       // per-lane singly linked list of entrants
    unsigned long long* head;  // [n_lanes] (tag << 32 | entrant) or stale
    int32_t* enter;       // [n_lanes], zeroed by k_lanescan after use
    int32_t* leave;       // [n_lanes], zeroed by k_lanescan after use
    Cand<Real>* cands;    // this step's lane-change candidates (cnt->n_cand of them)
    int32_t* cand_late;   // indices of the candidates k_lanescan resolves (cnt->n_late)
    unsigned long long* gap_head;  // [n_veh + n_lanes + 1] (tag << 32 | candidate) or stale
    unsigned long long* lane_tiles;
    int n_lane_tiles, max_slot_tiles, n_junc_chunks;
    int run_w;           // weight of a road-lane slot in k_decide's runs (junction-lane slot: 1); 0: fitted
    int4* runstat;       // [RUNSTAT_MAX] per k_decide work block: duration (ns, lo/hi), road-lane and junction-lane slots
    int cand_cap;        // lane-change candidates a k_decide block resolves itself (<= 256)
    Counters* cnt;       // this step's counters
    Counters* cnt_next;  // the next step's
    int* err;            // device error bits
    // ---- parameters
    Real dt, a_max, b_comf, T, s0, len, pol, a_th, b_safe, p_att, p_hi, p_lo, band;
    Real inv_2sqrt_ab;  // 1 / (2 sqrt(a b)), computed in double on the host
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85.
__device__ __forceinline__ void philox4x32_10(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                                              uint32_t c2, uint32_t c3, uint32_t out[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one widening multiply per product (high and low words together)
        const unsigned long long p0 = (unsigned long long)c0 * 0xD2511F53u;
        const unsigned long long p1 = (unsigned long long)c2 * 0xCD9E8D57u;
        const uint32_t n0 = uint32_t(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = uint32_t(p0 >> 32) ^ c3 ^ k1;
        c0 = n0; c1 = uint32_t(p1); c2 = n2; c3 = uint32_t(p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

template <typename Real>
__device__ __forceinline__ Real unit24(uint32_t w) {
    return Real(w >> 8) * Real(5.9604644775390625e-08);  // 2^-24, exact
}

template <typename Real> __device__ __forceinline__ Real rabs(Real x) { return x < Real(0) ? -x : x; }

// speed in units of 2^-24 m/s, rounded to nearest (for the speed metric).  In
// FP32 the product by 2^24 is exact and fits a 32-bit integer below 128 m/s,
// so no FP64 instruction is needed (FP64 throughput is low on this part).
__device__ __forceinline__ long long speed_fixed(float v) {
    return v < 128.0f ? (long long)__float2int_rn(v * 16777216.0f) : (long long)llrintf(v * 16777216.0f);
}
__device__ __forceinline__ long long speed_fixed(double v) { return (long long)llrint(v * 16777216.0); }

// x / y: IEEE division in FP64; the hardware's fast approximate division in
// FP32 (about 2 ulp, far inside the 1e-5 tolerance and the 1e-4 flag bands).
// Denominators here are desired speeds and gaps >= 1e-3 m, far from the
// range where the approximation degrades.
template <typename Real> __device__ __forceinline__ Real qdiv(Real x, Real y) { return x / y; }
#if !MOSS_IEEE_DIV
template <> __device__ __forceinline__ float qdiv<float>(float x, float y) { return __fdividef(x, y); }
#endif

// ---------------------------------------------------------------------------
// IDM, App. B.3 eqs. (1)-(2), delta = 4 as ((v/v0)^2)^2.
template <typename Real>
__device__ __forceinline__ Real idm_free(const Ctx<Real>& c, Real v, Real v0) {
    const Real r = qdiv(v, v0), r2 = r * r;
    return c.a_max * (Real(1) - r2 * r2);
}

template <typename Real>
__device__ __forceinline__ Real idm(const Ctx<Real>& c, Real v, Real v0, Real gap, Real dv) {
    const Real r = qdiv(v, v0), r2 = r * r;
    const Real dyn = v * c.T + v * dv * c.inv_2sqrt_ab;
    const Real sstar = c.s0 + (dyn > Real(0) ? dyn : Real(0));
    const Real g = gap > Real(1e-3) ? gap : Real(1e-3);
    const Real q = qdiv(sstar, g);
    return c.a_max * (Real(1) - r2 * r2 - q * q);
}

template <typename Real>
__device__ __forceinline__ Real p_lc(const Ctx<Real>& c, Real uT) {
    if (uT >= Real(1)) return c.p_hi;
    if (uT > Real(0)) return c.p_lo + (c.p_hi - c.p_lo) * uT;
    return c.p_lo;
}

// signal state of a junction at step t (§3.2 policies; reading R19)
__device__ __forceinline__ int junction_state(int policy, int manual, int offset, const int32_t* green,
                                              const int32_t* amber, int np, long long t) {
    if (policy == POL_NONE || np <= 0) return 512;
    if (policy == POL_MANUAL) return (manual & 15) | ((np & 15) << 4);
    long long cyc = 0;
    for (int p = 0; p < np; ++p) cyc += green[p] + amber[p];
    if (cyc <= 0) return 512;
    long long x = (t + offset) % cyc;
    if (x < 0) x += cyc;
    for (int p = 0; p < np; ++p) {
        const long long g = green[p], a = amber[p];
        if (x < g + a) return p | ((np & 15) << 4) | (x >= g ? 256 | (((p + 1) % np) << 10) : 0);
        x -= g + a;
    }
    return (np & 15) << 4;
}

// encoded state of a max-pressure junction (R23)
__device__ __forceinline__ int mp_encode(int4 m, int np) {
    return (m.x & 15) | ((np & 15) << 4) | (m.z >= 0 ? 256 | ((m.z & 15) << 10) : 0);
}

// signal state of junction j, `ahead` steps after its scenario's current step
// (a max-pressure junction: its current state)
template <typename Real>
__device__ __forceinline__ int junction_state_at(const Ctx<Real>& c, int j, int ahead) {
    const JuncInfo J = c.junc[j];
    const int pol = c.junc_policy[j], man = c.junc_manual[j];
    if (pol == POL_MAXP) return J.np > 0 ? mp_encode(c.mp[j], J.np) : 512;
    const long long t = c.scen_step[J.scen] + ahead;
    return junction_state(pol, man, J.offset, c.phase_green + J.phase_off, c.phase_amber + J.phase_off,
                          J.np, t);
}

// Max pressure (R23), one junction lane: adds its movement pressure (vehicles
// on the road lane it leaves minus vehicles on the road lane it feeds, in
// this step's snapshot) to the phases it is green in.
template <typename Real>
__device__ __forceinline__ void mp_accumulate(const Ctx<Real>& c, int k) {
    const int jl = c.jj_lane[k];
    const LaneInfo ji = c.lane[jl];
    if (ji.lo >= 0) return;  // a padding entry of a slot batch (names a road lane)
    if (c.junc_policy[ji.jb] != POL_MAXP || (ji.flags & LF_OFF) || c.scen_ctl[ji.scen]) return;
    const int from = c.jj_from[k], to = ji.hi;
    const int d = (c.cur.off[from + 1] - c.cur.off[from]) - (c.cur.off[to + 1] - c.cur.off[to]);
    if (d == 0) return;
#pragma unroll
    for (int ph = 0; ph < 8; ++ph)
        if ((ji.je >> ph) & 1) atomicAdd(&c.mp_press[ji.jb * 8 + ph], d);
}

// Max pressure (R23): advances junction j from this step to the next with the
// phase pressures of this step's snapshot (summed by mp_accumulate; cleared
// here for the next step) and returns the next step's state.  The phase is
// held for its programmed green; then the phase of maximal pressure is taken
// (the current one when it is maximal, else the smallest index), through the
// programmed amber.
template <typename Real>
__device__ __forceinline__ int mp_advance(const Ctx<Real>& c, int j) {
    const JuncInfo J = c.junc[j];
    int press[8];
    {
        int4* pp = reinterpret_cast<int4*>(c.mp_press + j * 8);
        const int4 a = pp[0], b = pp[1];
        pp[0] = make_int4(0, 0, 0, 0);
        pp[1] = make_int4(0, 0, 0, 0);
        press[0] = a.x; press[1] = a.y; press[2] = a.z; press[3] = a.w;
        press[4] = b.x; press[5] = b.y; press[6] = b.z; press[7] = b.w;
    }
    if (J.np <= 0) return 512;
    int4 m = c.mp[j];
    int p = m.x, e = m.y, q = m.z;
    if (q >= 0) {  // amber of p towards q
        if (e >= c.phase_amber[J.phase_off + p]) { p = q; q = -1; e = 1; }
        else e += 1;
    } else if (e >= c.phase_green[J.phase_off + p]) {
        int best = p, pb = press[0];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k == p) pb = press[k];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < J.np && press[k] > pb) { best = k; pb = press[k]; }
        if (best != p) {
            if (c.phase_amber[J.phase_off + p] > 0) { q = best; e = 1; }
            else { p = best; e = 1; }
        } else {
            e += 1;
        }
    } else {
        e += 1;
    }
    m.x = p; m.y = e; m.z = q;
    c.mp[j] = m;
    return mp_encode(m, J.np);
}

// light of a junction lane (its lane record ji) for this step
__device__ __forceinline__ int light_from(int st, const LaneInfo& ji) {
    if (st & 512) return LIGHT_GREEN;
    const int p = st & 15, mask = ji.je;
    if (!((mask >> p) & 1)) return LIGHT_RED;
    if (!(st & 256)) return LIGHT_GREEN;
    const int nx = (st >> 10) & 15;  // the phase after the amber
    return ((mask >> nx) & 1) ? LIGHT_GREEN : LIGHT_AMBER;
}

template <typename Real>
__device__ __forceinline__ int light_of(const Ctx<Real>& c, const LaneInfo& ji) {
    return light_from(c.junc_state[ji.jb], ji);
}

// junction lane leaving road lane (record li) towards road out_road (-1 if
// none); `hint` is tried first (the position of the matching junction lane of
// a neighbouring lane of the same road, usually the same)
// (junction lanes outside the road's current lane plan do not count, R28)
template <typename Real>
__device__ __forceinline__ int jl_toward(const Ctx<Real>& c, const LaneInfo& li, int out_road, int hint = -1) {
    if (hint >= 0 && li.jb + hint < li.je) {
        const LaneInfo x = c.lane[li.jb + hint];
        if (x.road == out_road && !(x.flags & LF_OFF)) return li.jb + hint;
    }
    for (int j = li.jb; j < li.je; ++j) {
        const LaneInfo x = c.lane[j];
        if (x.road == out_road && !(x.flags & LF_OFF)) return j;
    }
    return -1;
}

// (s_a, id_a) is ahead of (s_b, id_b) in lane order (R16)
template <typename Real>
__device__ __forceinline__ bool ahead(Real sa, int ia, Real sb, int ib) {
    return sa > sb || (sa == sb && ia < ib);
}

// first slot in [b, e) of the current snapshot that is NOT ahead of (s, id)
template <typename Real>
__device__ __forceinline__ int partition_point(const Ctx<Real>& c, int b, int e, Real s, int id) {
    int lo = b, hi = e;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const RecA<Real> m = c.cur.a[mid];
        if (ahead(m.s, m.id, s, id)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <typename Real>
struct LaneAcc {
    Real a, gap, stop_gap;
    int has_leader, stop, overlap, nl;  // nl: the next lane from this lane on the route
};

// Ego acceleration on a lane (record li) at (s, v): min over the leader (the
// vehicle at (ld_s, ld_v) in this lane if has_ld, else lookahead over at
// most two lanes, R11) and the stop line (R12).  nl: next lane from this
// lane on the ego's route (-1 none).
template <typename Real, bool Groups = true>
__device__ __forceinline__ LaneAcc<Real> accel_on_lane(const Ctx<Real>& c, const LaneInfo& li, Real s,
                                                       Real v, Real v0, bool has_ld, Real ld_s, Real ld_v,
                                                       int nl, int rptr, int rlast) {
    LaneAcc<Real> r;
    r.has_leader = 0; r.stop = 0; r.overlap = 0; r.gap = Real(0); r.stop_gap = Real(0); r.nl = nl;
    Real a = idm_free(c, v, v0);
    if (has_ld) {
        const Real gap = ld_s - c.len - s;
        a = idm(c, v, v0, gap, v - ld_v);
        r.has_leader = 1; r.gap = gap; r.overlap = gap < Real(0);
    }
    if (nl >= 0) {
        const LaneInfo ni = c.lane[nl];
        if (!has_ld) {
            Real base = Real(li.L) - s;
            int x = nl;
            LaneInfo xi = ni;
            for (int k = 0; k < 2; ++k) {
                const int b = c.cur.off[x], e = c.cur.off[x + 1];
                if (e > b) {
                    const RecA<Real> R = c.cur.a[e - 1];  // rearmost vehicle of lane x
                    const Real gap = base + R.s - c.len;
                    a = idm(c, v, v0, gap, v - R.v);
                    r.has_leader = 1; r.gap = gap;
                    break;
                }
                if (k == 1) break;
                base += Real(xi.L);
                // the lane after x on the route
                if (xi.lo < 0) {
                    x = xi.hi;  // junction lane -> its target road lane
                } else {
                    // x is a road lane (ego on a junction lane): the road after x's road
                    const int rp = rptr + 1;
                    x = (rp < rlast) ? jl_toward(c, xi, c.routes[rp + 1]) : -1;
                }
                if (x < 0) break;
                xi = c.lane[x];
            }
        }
        // stop line: a red or amber junction lane ahead (R12), or a next lane
        // restricted from passing (R25)
        if ((li.lo >= 0 && light_of(c, ni) != LIGHT_GREEN) || (ni.flags & LF_RESTRICTED)) {
            const Real gs = Real(li.L) - s;
            const Real as = idm(c, v, v0, gs, v);
            if (as < a) a = as;
            r.stop = 1; r.stop_gap = gs;
        }
    }
    // no junction lane from this road lane to the next road of the route
    // (lane groups, R27): stop at the lane end as before a red light
    if (Groups && nl < 0 && li.lo >= 0 && rptr < rlast) {
        const Real gs = Real(li.L) - s;
        const Real as = idm(c, v, v0, gs, v);
        if (as < a) a = as;
        r.stop = 1; r.stop_gap = gs;
    }
    r.a = a;
    return r;
}

// in-lane acceleration of a follower F (desired-speed factor f_v0f, lane limit
// vmax) towards a leader at (s_ld, v_ld), or on free road (politeness terms, R2)
template <typename Real>
__device__ __forceinline__ Real acc_pair(const Ctx<Real>& c, const RecA<Real>& F, float f_v0f, float vmax,
                                         bool has_ld, Real s_ld, Real v_ld) {
    const Real v0 = Real(f_v0f) * Real(vmax);
    if (!has_ld) return idm_free(c, F.v, v0);
    return idm(c, F.v, v0, s_ld - c.len - F.s, F.v - v_ld);
}

template <typename Real>
struct Decision {
    LaneAcc<Real> own;
    Real u, scale;
    int cand, dir, tl, TL, TF, flag;  // TL/TF: slots in the target lane or -1
    int nlt;                          // next lane on the route from the target lane
    int att;                          // MOBIL was evaluated (the attempt draw passed)
};

// The per-vehicle decision before conflict resolution (App. B.3), in two
// parts.  decide_own: the acceleration on the own lane and, on a road with
// two or more lanes, the MOBIL attempt draw (R4, R6).  decide_mobil: for a
// vehicle whose attempt draw passed, the MOBIL utilities of the sides, p_LC
// and the direction (R1-R5).  Both are pure functions of the snapshot.
template <typename Real>
struct OwnPart {
    LaneAcc<Real> own;
    float u_lc, u_dir;  // the draws for p_LC and the direction (exact in FP32)
    int att;            // the attempt draw passed: MOBIL is evaluated
    int mand;           // outside the lane group of the next road: mandatory change (R27)
};

// The neighbours in the own lane are the records of slots i - 1 and i + 1
// when their lane is the ego's (read with the ego's record, not after its
// lane's bounds).
template <typename Real, bool Groups = true>
__device__ __forceinline__ OwnPart<Real> decide_own(const Ctx<Real>& c, const RecA<Real>& E, const RecB& EB,
                                                    const LaneInfo& li, const RecA<Real>& OLr, long long t,
                                                    uint32_t k0, uint32_t k1, int vbase) {
    OwnPart<Real> P;
    P.att = 0; P.mand = 0; P.u_lc = 0.0f; P.u_dir = 0.0f;
    P.own = accel_on_lane<Real, Groups>(c, li, E.s, E.v, Real(EB.v0f) * Real(li.vmax), OLr.lane == E.lane, OLr.s,
                                        OLr.v, EB.nl, EB.rptr, EB.rlast);
    if (li.lo < 0 || li.hi - li.lo < 2) return P;  // junction lane or single-lane road
    // no access to the next road from this lane: a mandatory change, no draw (R27)
    if (Groups && EB.nl < 0 && EB.rptr < EB.rlast) { P.mand = 1; return P; }
    uint32_t w[4];
    philox4x32_10(k0, k1, uint32_t(E.id - vbase), uint32_t(t), 0u, 0u, w);
    const Real u_att = unit24<Real>(w[0]);
    if (!(u_att < c.p_att)) return P;
    P.att = 1;
    P.u_lc = unit24<float>(w[1]);
    P.u_dir = unit24<float>(w[2]);
    return P;
}

template <typename Real, bool Groups = true>
__device__ __forceinline__ Decision<Real> decide_mobil(const Ctx<Real>& c, const RecA<Real>& E, const RecB& EB,
                                                       const LaneInfo& li, const RecA<Real>& OLr,
                                                       const RecA<Real>& OFr, float of_v0f,
                                                       const LaneAcc<Real>& own, float f_lc, float f_dir) {
    Decision<Real> D;
    D.cand = 0; D.dir = 0; D.tl = -1; D.TL = -1; D.TF = -1; D.flag = 0; D.nlt = -1; D.att = 1;
    D.u = Real(0); D.scale = Real(1);
    D.own = own;
    const int lane = E.lane;
    const Real v0f = Real(EB.v0f);
    const Real u_lc = Real(f_lc), u_dir = Real(f_dir);

    Real a_old = Real(0), at_old = Real(0);
    if (OFr.lane == lane) {
        a_old = acc_pair(c, OFr, of_v0f, li.vmax, true, E.s, E.v);
        if (OLr.lane == lane) {
            at_old = acc_pair(c, OFr, of_v0f, li.vmax, true, OLr.s, OLr.v);
        } else {
            at_old = acc_pair(c, OFr, of_v0f, li.vmax, false, Real(0), Real(0));
        }
    }
    // next road of the route (for the target lane's junction lane)
    const int next_road = (EB.nl >= 0) ? c.lane[EB.nl].road : -1;
    // The sides that exist are visited in order, so every vehicle with one
    // side (an edge lane) runs the first pass together with its warp
    // neighbours, whichever side that is; results go to the left/right
    // variables by select.  Same arithmetic per side as a fixed left/right
    // loop: the decision does not depend on the visiting order.
    Real u0 = Real(0), u1 = Real(0), scl0 = Real(0), scl1 = Real(0);
    int feas0 = 0, feas1 = 0, TL0 = -1, TL1 = -1, TF0 = -1, TF1 = -1, NL0 = -1, NL1 = -1;
    const Real pos_scale = E.s > Real(1) ? E.s : Real(1);
    // a side is a lane of the road that is not restricted from passing (R25)
    const int has_l = lane - 1 >= li.lo && !(c.lane[lane - 1].flags & LF_RESTRICTED);
    const int has_r = lane + 1 < li.hi && !(c.lane[lane + 1].flags & LF_RESTRICTED);
    const int n_sides = has_l + has_r;
#pragma unroll 1
    for (int k = 0; k < n_sides; ++k) {
        const int side = (k == 0 && has_l) ? 0 : 1;
        const int tl = side == 0 ? lane - 1 : lane + 1;
        const LaneInfo ti = c.lane[tl];
        // next lane from the target lane; a lane without access to the next
        // road is outside the vehicle's group: not a side (R27)
        const int nlt = (next_road >= 0) ? jl_toward(c, ti, next_road, EB.nl - li.jb) : -1;
        if (Groups && next_road >= 0 && nlt < 0) continue;
        const int tb = c.cur.off[tl], te = c.cur.off[tl + 1];
        const int p = partition_point(c, tb, te, E.s, E.id);
        const int TL = (p > tb) ? p - 1 : -1, TF = (p < te) ? p : -1;
        int ok = 1;
        RecA<Real> TLr, TFr;
        TLr.s = Real(0); TLr.v = Real(0); TFr.s = Real(0); TFr.v = Real(0);
        if (TL >= 0) {
            TLr = c.cur.a[TL];
            const Real g = TLr.s - c.len - E.s;
            if (!(g > Real(0))) ok = 0;
            if (rabs(g) < c.band * pos_scale) D.flag = 1;
        }
        if (TF >= 0) {
            TFr = c.cur.a[TF];
            const Real g = E.s - c.len - TFr.s;
            if (!(g > Real(0))) ok = 0;
            if (rabs(g) < c.band * pos_scale) D.flag = 1;
        }
        const Real at_ego =
            accel_on_lane<Real, Groups>(c, ti, E.s, E.v, v0f * Real(ti.vmax), TL >= 0, TLr.s, TLr.v, nlt, EB.rptr,
                                        EB.rlast).a;
        Real a_new = Real(0), at_new = Real(0);
        if (TF >= 0) {
            const float fv0f = c.cur.b[TF].v0f;
            a_new = acc_pair(c, TFr, fv0f, ti.vmax, TL >= 0, TLr.s, TLr.v);
            at_new = acc_pair(c, TFr, fv0f, ti.vmax, true, E.s, E.v);
            if (!(at_new >= -c.b_safe)) ok = 0;
            const Real sc = rabs(at_new) > Real(1) ? rabs(at_new) : Real(1);
            if (rabs(at_new + c.b_safe) < c.band * sc) D.flag = 1;
        }
        const Real us = (at_ego - D.own.a) + c.pol * ((at_new - a_new) + (at_old - a_old)) - c.a_th;
        const Real ss = rabs(at_ego) + rabs(D.own.a) +
                        c.pol * (rabs(at_new) + rabs(a_new) + rabs(at_old) + rabs(a_old)) + c.a_th;
        if (side == 0) { u0 = us; scl0 = ss; feas0 = ok; TL0 = TL; TF0 = TF; NL0 = nlt; }
        else           { u1 = us; scl1 = ss; feas1 = ok; TL1 = TL; TF1 = TF; NL1 = nlt; }
    }
    const Real u[2] = {u0, u1}, scl[2] = {scl0, scl1};
    const int feas[2] = {feas0, feas1}, TLs[2] = {TL0, TL1}, TFs[2] = {TF0, TF1}, NLs[2] = {NL0, NL1};
    Real scale = Real(1);
    for (int sd = 0; sd < 2; ++sd)
        if (feas[sd] && scl[sd] > scale) scale = scl[sd];
    D.scale = scale;
    const Real uLp = (feas[0] && u[0] > Real(0)) ? u[0] : Real(0);
    const Real uRp = (feas[1] && u[1] > Real(0)) ? u[1] : Real(0);
    const Real uT = uLp + uRp;
    const Real pl = p_lc(c, uT);
    const Real band_p = (uT < Real(1) + c.band * scale) ? c.band * scale : c.band;
    if (rabs(u_lc - pl) < band_p) D.flag = 1;
    if (!(u_lc < pl)) return D;
    int side = -1;
    if (uT > Real(0)) {
        const Real q = uLp - u_dir * uT;
        if (rabs(q) < c.band * scale) D.flag = 1;
        if (uT < c.band * scale) D.flag = 1;
        side = q > Real(0) ? 0 : 1;
    } else {
        if (feas[0] && feas[1]) side = u_dir < Real(0.5) ? 0 : 1;
        else if (feas[0]) side = 0;
        else if (feas[1]) side = 1;
        if (side >= 0 && uT < c.band * scale) D.flag = 1;
    }
    if (side < 0) return D;
    D.cand = 1;
    D.dir = side == 0 ? -1 : 1;
    D.tl = side == 0 ? lane - 1 : lane + 1;
    D.TL = TLs[side]; D.TF = TFs[side]; D.nlt = NLs[side];
    D.u = u[side];
    return D;
}

// Mandatory change (R27) of a vehicle outside the lane group of its next
// road: one lane towards the nearest lane of the group (ties: left) when the
// safety part of R2 holds (gaps > 0, ã_new >= -b_safe); no random draw; in
// the conflict rule R9 its utility is MAND_U, above any discretionary one.
constexpr double MAND_U = 1e30;

template <typename Real>
__device__ __forceinline__ Decision<Real> decide_mandatory(const Ctx<Real>& c, int i, const RecA<Real>& E,
                                                           const RecB& EB, const LaneInfo& li,
                                                           const LaneAcc<Real>& own) {
    Decision<Real> D;
    D.cand = 0; D.dir = 0; D.tl = -1; D.TL = -1; D.TF = -1; D.flag = 0; D.nlt = -1; D.att = 0;
    D.u = Real(0); D.scale = Real(1);
    D.own = own;
    const int lane = E.lane;
    const int next_road = c.routes[EB.rptr + 1];
    int best = -1;
    for (int k = li.lo; k < li.hi; ++k) {
        if (jl_toward(c, c.lane[k], next_road) < 0) continue;
        const int dk = k > lane ? k - lane : lane - k, db = best > lane ? best - lane : lane - best;
        if (best < 0 || dk < db) best = k;
    }
    if (best < 0) return D;
    const int dir = best < lane ? -1 : 1, tl = lane + dir;
    const LaneInfo ti = c.lane[tl];
    if (ti.flags & LF_RESTRICTED) return D;
    const int tb = c.cur.off[tl], te = c.cur.off[tl + 1];
    const int p = partition_point(c, tb, te, E.s, E.id);
    const int TL = (p > tb) ? p - 1 : -1, TF = (p < te) ? p : -1;
    const Real pos_scale = E.s > Real(1) ? E.s : Real(1);
    int ok = 1;
    if (TL >= 0) {
        const RecA<Real> T = c.cur.a[TL];
        const Real g = T.s - c.len - E.s;
        if (!(g > Real(0))) ok = 0;
        if (rabs(g) < c.band * pos_scale) D.flag = 1;
    }
    if (TF >= 0) {
        const RecA<Real> F = c.cur.a[TF];
        const Real g = E.s - c.len - F.s;
        if (!(g > Real(0))) ok = 0;
        if (rabs(g) < c.band * pos_scale) D.flag = 1;
        const Real at_new = acc_pair(c, F, c.cur.b[TF].v0f, ti.vmax, true, E.s, E.v);
        if (!(at_new >= -c.b_safe)) ok = 0;
        const Real sc = rabs(at_new) > Real(1) ? rabs(at_new) : Real(1);
        if (rabs(at_new + c.b_safe) < c.band * sc) D.flag = 1;
    }
    if (!ok) return D;
    D.cand = 1; D.dir = dir; D.tl = tl; D.TL = TL; D.TF = TF;
    D.nlt = jl_toward(c, ti, next_road);
    D.u = Real(MAND_U);
    D.scale = Real(1);
    return D;
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long load_acquire(unsigned long long* p) {
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*p);
    return a.load(cuda::memory_order_acquire);
}
// look-back words carry flag and value in one 64-bit word, so a relaxed
// (single-copy atomic) load that sees the flag also sees the value
__device__ __forceinline__ unsigned long long load_relaxed(unsigned long long* p) {
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*p);
    return a.load(cuda::memory_order_relaxed);
}
__device__ __forceinline__ void store_release(unsigned long long* p, unsigned long long v) {
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*p);
    a.store(v, cuda::memory_order_release);
}

// Slot in an array shared through one counter: the threads of the warp that
// are here together take consecutive slots with one atomic.
__device__ __forceinline__ int warp_claim(int* counter) {
    const unsigned m = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(m, base, leader);
    return base + __popc(m & ((1u << lane) - 1u));
}

// Warp-cooperative look-back of a decoupled scan (all 32 lanes of one warp).
// Tile words: flag (2 bits: 1 aggregate, 2 inclusive prefix) | 62-bit value.
// Returns the exclusive prefix of `tile`; sets *timeout if a bounded wait gave up.
__device__ __forceinline__ unsigned long long warp_lookback(unsigned long long* st, int tile, bool* timeout) {
    const int lane = threadIdx.x & 31;
    unsigned long long prefix = 0;
    int p = tile - 1;
    long long spins = 0;
    while (p >= 0) {
        const int idx = p - lane;
        const unsigned long long w = idx >= 0 ? load_relaxed(&st[idx]) : (2ull << 62);
        const unsigned f = (unsigned)(w >> 62);
        const unsigned m2 = __ballot_sync(0xffffffffu, f == 2);
        const unsigned m0 = __ballot_sync(0xffffffffu, f == 0);
        const int first2 = m2 ? __ffs(m2) - 1 : 31;
        const unsigned upto = first2 >= 31 ? 0xffffffffu : ((2u << first2) - 1u);
        if (m0 & upto) {
            if (++spins > SPIN_LIMIT) { *timeout = true; return prefix; }
            if (spins > 16) __nanosleep(64);
            continue;
        }
        unsigned long long val = (lane <= first2) ? (w & ((1ull << 62) - 1)) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
        prefix += val;
        if (m2) break;
        p -= 32;
    }
    return prefix;
}

// Per-scenario metric accumulation: register partials per thread, flushed
// with one set of atomics per block when the whole block shares a scenario.
// Counts are 32-bit (each is at most the number of vehicles the thread
// handles in one launch); travel-time and speed sums are 64-bit.
constexpr int MACC_N = 8;
struct MetricAcc {
    int scen;
    int upd, arr, lc, flg, ovl, mob;  // updates, arrived, lane changes, flagged, overlaps, MOBIL evaluations
    long long tt, spd;                // travel time in steps, speed in units of 2^-24 m/s
};

__device__ __forceinline__ int metric_field(int k) {
    switch (k) {
        case 0: return M_UPDATES;
        case 1: return M_ARRIVED;
        case 2: return M_TT_STEPS;
        case 3: return M_SPEED_FX;
        case 4: return M_LANE_CHANGES;
        case 5: return M_FLAGGED;
        case 6: return M_OVERLAPS;
        default: return M_MOBIL;
    }
}

__device__ __forceinline__ long long macc_value(const MetricAcc& a, int k) {
    switch (k) {
        case 0: return a.upd;
        case 1: return a.arr;
        case 2: return a.tt;
        case 3: return a.spd;
        case 4: return a.lc;
        case 5: return a.flg;
        case 6: return a.ovl;
        default: return a.mob;
    }
}

__device__ __forceinline__ void macc_reset(MetricAcc& a, int scen) {
    a.scen = scen;
    a.upd = a.arr = a.lc = a.flg = a.ovl = a.mob = 0;
    a.tt = a.spd = 0;
}

__device__ __forceinline__ void macc_flush_thread(MetricAcc& a, long long* metrics) {
    if (a.scen < 0) return;
#pragma unroll
    for (int k = 0; k < MACC_N; ++k) {
        const long long x = macc_value(a, k);
        if (x) atomicAdd((unsigned long long*)&metrics[a.scen * M_NFIELDS + metric_field(k)], (unsigned long long)x);
    }
}

// Block-level flush: reduce in shared memory when every thread holds the
// same scenario (or nothing), else fall back to per-thread atomics.
template <int THREADS>
__device__ void macc_flush_block(MetricAcc& a, long long* metrics) {
    __shared__ long long red[MACC_N][THREADS / 32];
    __shared__ int scen0;
    const int tid = threadIdx.x;
    if (tid == 0) scen0 = -1;
    __syncthreads();
    if (a.scen >= 0) atomicMax(&scen0, a.scen);
    __syncthreads();
    const int s0 = scen0;
    const bool uniform = __syncthreads_and(a.scen < 0 || a.scen == s0);
    if (!uniform) { macc_flush_thread(a, metrics); return; }
    if (s0 < 0) return;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < MACC_N; ++k) {
        long long x = a.scen < 0 ? 0 : macc_value(a, k);
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][warp] = x;
    }
    __syncthreads();
    if (tid < MACC_N) {
        long long x = 0;
        for (int w = 0; w < THREADS / 32; ++w) x += red[tid][w];
        if (x) atomicAdd((unsigned long long*)&metrics[s0 * M_NFIELDS + metric_field(tid)], (unsigned long long)x);
    }
}

}  // namespace moss
