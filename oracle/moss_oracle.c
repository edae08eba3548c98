/*
 * FP64 CPU ORACLE for the per-timestep microscopic vehicle update.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (arxiv 2406.10661):
 *   - two-phase step: every vehicle reads only the previous step's snapshot and
 *     writes only its own runtime state (§3.1 "Two-phase Parallel Process for
 *     Read/Write Separation"; App. B.2 prepare/update phases);
 *   - neighbour sensing: the leader/follower on the own lane and on the
 *     adjacent lanes, and the first vehicle of the next lane when the own lane
 *     has no leader (§3.1 "Linked-list based Vehicle Sensing Indexes";
 *     App. B.3).  The oracle uses the plain definition, a linear scan over the
 *     lane's vehicles, with no index structure;
 *   - IDM car following, App. B.3 equations (1)-(2), delta = 4;
 *   - randomized MOBIL: utility u, u_T = max(0,u_L)+max(0,u_R) and the
 *     piecewise p_LC (App. B.3);
 *   - red/amber stop in front of the next lane's signal (App. B.3, last
 *     paragraph), fixed-time / manual / no signal policies (§3.2);
 *   - lane transfer at the lane end, arrival handling and departure insertion
 *     (App. B.2 prepare stream 3, update streams 1 and 3);
 *   - metrics: throughput, average travelling time, network speed (§3.3).
 *
 * Where the paper is silent or garbled the oracle follows these readings
 * (shared with the CUDA path, listed with reasons in the design notes):
 *   R1  MOBIL tilde = acceleration AFTER the change (standard MOBIL; the
 *       paper's wording is reversed relative to its own formula).
 *   R2  u_d = (ã_ego - a_ego) + p((ã_new - a_new) + (ã_old - a_old)) - a_th;
 *       side d is feasible iff its lane exists on the road, the gaps to the
 *       target leader and target follower are > 0, and ã_new >= -b_safe.
 *       Politeness terms use in-lane car following only (no lookahead, no
 *       stop line); a missing follower contributes 0.
 *   R3  p_LC = p_lo + (p_hi - p_lo) u_T for 0 < u_T < 1 (continuous reading of
 *       the garbled middle branch); p_hi for u_T >= 1; p_lo for u_T = 0.
 *   R4  MOBIL is evaluated only when the attempt draw u_att < p_attempt.
 *   R5  direction: u_T > 0 -> left iff u_dir * u_T < max(0,u_L); u_T = 0 ->
 *       uniform over feasible sides (left iff u_dir < 0.5 when both).
 *   R6  Philox4x32-10, key (seed lo, seed hi ^ scenario), counter (vehicle
 *       id, step, 0, 0); words 0,1,2 -> u_att, u_lc, u_dir = (w >> 8) 2^-24.
 *   R7  lane changes only on road lanes of roads with >= 2 lanes; the change
 *       is instantaneous at the end of the step and keeps s.
 *   R9  conflict: two granted candidates entering the same lane from opposite
 *       sides into the same snapshot gap (same target leader and follower):
 *       the larger u wins, ties to the smaller id; losers keep their lane.
 *   R10 v0 = v0f * speed limit of the lane.
 *   R11 lookahead: with no leader on the lane, the rearmost vehicle of the
 *       next lane on the route, else of the lane after it (at most 2 lanes).
 *   R12 red/amber: IDM against a standing obstacle at the lane end (gap L-s,
 *       dv = v).  Ballistic update: v' = max(0, v + a dt); d = v dt + a dt^2/2
 *       if v + a dt >= 0, else v^2 / (-2a).
 *   R13 clamp: d <= max(0, gap to the leader used), d <= max(0, L - s) when
 *       the stop line is active; IDM uses max(gap, 1e-3).
 *   R16 lane order: s descending, ties by smaller id first.
 *   R17 transfer while s' > L (arrival on the last road when s' >= L).
 *   R18 insertion at s = 0, v = 0, one per start lane per step, FIFO by
 *       (departure, id), when the lane is empty or its rearmost vehicle has
 *       s - len >= s0 (snapshot).
 *   R19 fixed time: phase p green for green[p] steps then amber for amber[p]
 *       steps, cycle shifted by the junction offset; a lane green in phase p
 *       and also in phase p+1 stays green through p's amber.  Manual: the set
 *       phase is green, no amber.  None: always green.
 *   R21 metrics: network speed = sum of post-update speeds over all vehicle
 *       updates / number of vehicle updates; ATT = mean (arrival time -
 *       departure time) over finished trips.
 *   R22 a decision whose deciding quantity is within flag_band (scaled) of
 *       its threshold is flagged.
 *   R23 max pressure (§3.2 MAX_PRESSURE policy; App. B.2 prepare stream 1 /
 *       update stream 2; Varaiya 2013): the pressure of a movement (a
 *       junction lane) is the number of vehicles on the road lane it leaves
 *       minus the number on the road lane it feeds, counted in the step's
 *       snapshot; the pressure of a phase is the sum over the junction lanes
 *       green in it.  A junction holds its phase for at least the phase's
 *       programmed green time; from then on, at the end of every step it
 *       takes the phase of maximal pressure (its current phase when that one
 *       is maximal, else the smallest index among the maxima) for the next
 *       step.  A change of phase goes through the current phase's programmed
 *       amber (lanes green in both phases stay green, as in R19).  Setting
 *       the policy starts the phase the junction shows at that step, green.
 *   R24 metrics of §3.3: the queue length of a lane counts the vehicles with
 *       v < 0.1 m/s whose distance to the lane end L - s is at most 50 m; the
 *       average vehicle speed of a road is the mean speed of the vehicles on
 *       its lanes, or the mean speed limit of its lanes when it is empty.
 *   R25 lane setters (§3.2 "Lane"): a new maximum speed applies from the next
 *       step (v0 = v0f x limit, R10).  A lane restricted from passing is not
 *       entered: a vehicle whose next lane is restricted stops at the end of
 *       its lane as before a red light (R12, R13); MOBIL treats a restricted
 *       adjacent lane as absent; no departure is inserted onto it.  Vehicles
 *       already on it drive on.
 *   R26 re-routing (§3.2 "Vehicle", set_vehicle_route): the new route starts
 *       with the road the vehicle is on (a waiting vehicle: the road of its
 *       start lane; on a junction lane: the road it is entering, the road
 *       just left is kept in front), consecutive roads must be joined by a
 *       junction lane, and the vehicle arrives at the end of the new route's
 *       last road as every trip does.
 *   R27 lane groups (App. B.3: vehicles may not change lanes away from the
 *       group of lanes that gives access to the next road): the group of a
 *       vehicle is the set of lanes of its road with a junction lane to the
 *       next road of its route.  Inside the group, MOBIL treats an adjacent
 *       lane outside it as absent.  Outside the group (it entered the road
 *       on a lane without access), the vehicle cannot leave the road from its
 *       lane: it stops at the lane end as before a red light, and it changes
 *       one lane towards the nearest lane of the group (ties: left) whenever
 *       the safety part of R2 holds for that lane (gaps > 0, ã_new >=
 *       -b_safe) — a mandatory change, without random draws, entered in the
 *       conflict rule R9 with utility U_MAND (larger than any discretionary
 *       utility).  On the last road of the route there is no group.
 *   R28 lane plans (§3.2 "Road", set_road_lane_plan): every junction lane
 *       belongs to a set of plans (bit p of its plan mask); a road uses one
 *       plan at a time (plan 0 at the start).  A junction lane outside the
 *       current plan of its road is not used: no lane has access through it
 *       (R27), nobody enters it, and it adds no pressure (R23).  Vehicles
 *       already on it drive on.  A plan change applies from the next step.
 */
#define U_MAND 1e30
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the
 * published round definition: two 32x32->64 multiplies per round with
 * multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 /
 * 0xBB67AE85, ten rounds.                                                    */
void mo_philox4x32_10(uint32_t k0, uint32_t k1, const uint32_t ctr_in[4], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double unit24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
enum { LIGHT_GREEN = 0, LIGHT_AMBER = 1, LIGHT_RED = 2 };
enum { POLICY_FIXED = 0, POLICY_MANUAL = 1, POLICY_NONE = 2, POLICY_MAXP = 3 };
enum { ST_WAITING = 0, ST_ACTIVE = 1, ST_ARRIVED = 2 };
enum {
    F_FLAGGED = 1, F_CHANGED = 2, F_CANDIDATE = 4, F_TRANSFER = 8,
    F_ARRIVED = 16, F_INSERTED = 32, F_CONFLICT_LOST = 64
};

typedef struct {
    /* network */
    int n_roads, n_road_lanes, n_lanes, n_junctions;
    int *road_lane_off, *lane_road;
    double *L, *vmax;
    int *jl_off;                       /* [n_road_lanes+1] */
    int *jl_target, *jl_junction, *jl_mask; /* indexed by absolute lane id */
    int *junc_offset, *junc_phase_off, *phase_green, *phase_amber;
    int *junc_policy, *junc_manual;
    int *jl_from;                      /* road lane a junction lane leaves (absolute ids) */
    int *mp_phase, *mp_elapsed, *mp_pending; /* max-pressure state per junction (R23) */
    int *restricted;                   /* per lane: restricted from passing (R25) */
    int *jl_plans, *road_plan;         /* R28: plan mask per lane (junction lanes), plan per road */
    /* vehicles */
    int n_veh;
    int *route_beg, *route_len, *routes, *start_lane, *dep;  /* route of vid: routes[beg .. beg+len) */
    long routes_used, routes_cap;
    double *v0f;
    /* runtime state */
    int *status, *lane, *rc, *flags;
    double *s, *v;
    /* insertion FIFOs per road lane */
    int *q_off, *q_ids, *q_head;
    /* parameters */
    double dt, a_max, b_comf, T, s0, delta, len, pol, a_th, b_safe, p_att, p_hi, p_lo, band;
    uint32_t key0, key1;
    long step;
    int reverse_order;
    /* metrics */
    double m_speed_sum, m_tt_sum;
    long m_updates, m_arrived, m_lane_changes, m_flagged, m_overlaps, m_inserted, m_errors;
    long m_mobil;
} Oracle;

/* Snapshot of the public state at the start of a step (§3.1). */
typedef struct {
    int n;
    char *active;
    int *lane, *rc;
    double *s, *v;
    int *lane_cnt, *lane_first, *members; /* unordered member list per lane */
    int *light;                           /* per absolute lane id (junction lanes) */
} Snap;

static void* xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

/* junction lane j is part of the current plan of the road it leaves (R28) */
static int jl_available(const Oracle* O, int j) {
    return (O->jl_plans[j] >> O->road_plan[O->lane_road[O->jl_from[j]]]) & 1;
}


/* ------------------------------------------------------------------------ */
/* Creation                                                                   */
void* mo_create(int n_roads, const int* road_lane_off, int n_lanes, int n_road_lanes,
                const float* lane_length, const float* lane_vmax, const int* jl_off,
                const int* jl_target, const int* jl_junction, const int* jl_mask,
                int n_junctions, const int* junc_offset, const int* junc_phase_off,
                const int* phase_green, const int* phase_amber, int n_veh,
                const int* route_off, const int* routes, const int* start_lane,
                const int* dep, const float* v0f, const double* prm,
                unsigned long long seed, unsigned int scenario) {
    Oracle* O = (Oracle*)xcalloc(1, sizeof(Oracle));
    O->n_roads = n_roads; O->n_lanes = n_lanes; O->n_road_lanes = n_road_lanes;
    O->n_junctions = n_junctions; O->n_veh = n_veh;
    O->road_lane_off = (int*)xcalloc(n_roads + 1, sizeof(int));
    memcpy(O->road_lane_off, road_lane_off, sizeof(int) * (n_roads + 1));
    O->lane_road = (int*)xcalloc(n_lanes, sizeof(int));
    for (int l = 0; l < n_lanes; ++l) O->lane_road[l] = -1;
    for (int r = 0; r < n_roads; ++r)
        for (int l = road_lane_off[r]; l < road_lane_off[r + 1]; ++l) O->lane_road[l] = r;
    O->L = (double*)xcalloc(n_lanes, sizeof(double));
    O->vmax = (double*)xcalloc(n_lanes, sizeof(double));
    for (int l = 0; l < n_lanes; ++l) { O->L[l] = lane_length[l]; O->vmax[l] = lane_vmax[l]; }
    O->jl_off = (int*)xcalloc(n_road_lanes + 1, sizeof(int));
    memcpy(O->jl_off, jl_off, sizeof(int) * (n_road_lanes + 1));
    O->jl_target = (int*)xcalloc(n_lanes, sizeof(int));
    O->jl_junction = (int*)xcalloc(n_lanes, sizeof(int));
    O->jl_mask = (int*)xcalloc(n_lanes, sizeof(int));
    for (int l = 0; l < n_lanes; ++l) { O->jl_target[l] = -1; O->jl_junction[l] = -1; }
    for (int l = n_road_lanes; l < n_lanes; ++l) {
        O->jl_target[l] = jl_target[l - n_road_lanes];
        O->jl_junction[l] = jl_junction[l - n_road_lanes];
        O->jl_mask[l] = jl_mask[l - n_road_lanes];
    }
    O->junc_offset = (int*)xcalloc(n_junctions, sizeof(int));
    O->junc_phase_off = (int*)xcalloc(n_junctions + 1, sizeof(int));
    O->junc_policy = (int*)xcalloc(n_junctions, sizeof(int));
    O->junc_manual = (int*)xcalloc(n_junctions, sizeof(int));
    if (n_junctions) memcpy(O->junc_offset, junc_offset, sizeof(int) * n_junctions);
    memcpy(O->junc_phase_off, junc_phase_off, sizeof(int) * (n_junctions + 1));
    int np = junc_phase_off[n_junctions];
    O->phase_green = (int*)xcalloc(np, sizeof(int));
    O->phase_amber = (int*)xcalloc(np, sizeof(int));
    if (np) {
        memcpy(O->phase_green, phase_green, sizeof(int) * np);
        memcpy(O->phase_amber, phase_amber, sizeof(int) * np);
    }
    for (int j = 0; j < n_junctions; ++j)
        O->junc_policy[j] = (junc_phase_off[j + 1] > junc_phase_off[j]) ? POLICY_FIXED : POLICY_NONE;
    O->jl_from = (int*)xcalloc(n_lanes, sizeof(int));
    for (int l = 0; l < n_lanes; ++l) O->jl_from[l] = -1;
    for (int l = 0; l < n_road_lanes; ++l)
        for (int jl = jl_off[l]; jl < jl_off[l + 1]; ++jl) O->jl_from[jl] = l;
    O->mp_phase = (int*)xcalloc(n_junctions, sizeof(int));
    O->mp_elapsed = (int*)xcalloc(n_junctions, sizeof(int));
    O->mp_pending = (int*)xcalloc(n_junctions, sizeof(int));
    O->restricted = (int*)xcalloc(n_lanes, sizeof(int));
    O->jl_plans = (int*)xcalloc(n_lanes, sizeof(int));
    for (int l = 0; l < n_lanes; ++l) O->jl_plans[l] = 0xff;
    O->road_plan = (int*)xcalloc(n_roads, sizeof(int));

    O->route_beg = (int*)xcalloc(n_veh, sizeof(int));
    O->route_len = (int*)xcalloc(n_veh, sizeof(int));
    for (int i = 0; i < n_veh; ++i) { O->route_beg[i] = route_off[i]; O->route_len[i] = route_off[i + 1] - route_off[i]; }
    O->routes_used = route_off[n_veh];
    O->routes_cap = route_off[n_veh] > 0 ? route_off[n_veh] : 1;
    O->routes = (int*)xcalloc(O->routes_cap, sizeof(int));
    memcpy(O->routes, routes, sizeof(int) * route_off[n_veh]);
    O->start_lane = (int*)xcalloc(n_veh, sizeof(int));
    O->dep = (int*)xcalloc(n_veh, sizeof(int));
    O->v0f = (double*)xcalloc(n_veh, sizeof(double));
    memcpy(O->start_lane, start_lane, sizeof(int) * n_veh);
    memcpy(O->dep, dep, sizeof(int) * n_veh);
    for (int i = 0; i < n_veh; ++i) O->v0f[i] = v0f[i];
    O->status = (int*)xcalloc(n_veh, sizeof(int));
    O->lane = (int*)xcalloc(n_veh, sizeof(int));
    O->rc = (int*)xcalloc(n_veh, sizeof(int));
    O->flags = (int*)xcalloc(n_veh, sizeof(int));
    O->s = (double*)xcalloc(n_veh, sizeof(double));
    O->v = (double*)xcalloc(n_veh, sizeof(double));
    for (int i = 0; i < n_veh; ++i) { O->status[i] = ST_WAITING; O->lane[i] = -1; }

    /* FIFO per start lane, ordered by (departure step, id) (R18). */
    O->q_off = (int*)xcalloc(n_road_lanes + 1, sizeof(int));
    O->q_head = (int*)xcalloc(n_road_lanes, sizeof(int));
    O->q_ids = (int*)xcalloc(n_veh, sizeof(int));
    for (int i = 0; i < n_veh; ++i) O->q_off[start_lane[i] + 1]++;
    for (int l = 0; l < n_road_lanes; ++l) O->q_off[l + 1] += O->q_off[l];
    int* fill = (int*)xcalloc(n_road_lanes, sizeof(int));
    for (int i = 0; i < n_veh; ++i) {
        int l = start_lane[i];
        O->q_ids[O->q_off[l] + fill[l]++] = i;
    }
    free(fill);
    for (int l = 0; l < n_road_lanes; ++l) {   /* insertion sort by (dep, id) */
        for (int a = O->q_off[l] + 1; a < O->q_off[l + 1]; ++a) {
            int x = O->q_ids[a], b = a - 1;
            while (b >= O->q_off[l] && (O->dep[O->q_ids[b]] > O->dep[x] ||
                   (O->dep[O->q_ids[b]] == O->dep[x] && O->q_ids[b] > x))) {
                O->q_ids[b + 1] = O->q_ids[b];
                --b;
            }
            O->q_ids[b + 1] = x;
        }
        O->q_head[l] = O->q_off[l];
    }

    O->dt = prm[0]; O->a_max = prm[1]; O->b_comf = prm[2]; O->T = prm[3]; O->s0 = prm[4];
    O->delta = prm[5]; O->len = prm[6]; O->pol = prm[7]; O->a_th = prm[8];
    O->b_safe = prm[9]; O->p_att = prm[10]; O->p_hi = prm[11]; O->p_lo = prm[12];
    O->band = prm[13];
    O->key0 = (uint32_t)(seed & 0xffffffffull);
    O->key1 = (uint32_t)(seed >> 32) ^ (uint32_t)scenario;
    return O;
}

void mo_destroy(void* h) {
    Oracle* O = (Oracle*)h;
    if (!O) return;
    void* ptrs[] = {O->road_lane_off, O->lane_road, O->L, O->vmax, O->jl_off, O->jl_target,
                    O->jl_junction, O->jl_mask, O->junc_offset, O->junc_phase_off,
                    O->phase_green, O->phase_amber, O->junc_policy, O->junc_manual,
                    O->jl_from, O->mp_phase, O->mp_elapsed, O->mp_pending, O->restricted, O->jl_plans, O->road_plan, O->route_beg, O->route_len, O->routes, O->start_lane, O->dep, O->v0f, O->status,
                    O->lane, O->rc, O->flags, O->s, O->v, O->q_off, O->q_ids, O->q_head};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
    free(O);
}

/* ------------------------------------------------------------------------ */
/* Signals (§3.2 policies; reading R19)                                       */
/* phase of junction j's fixed-time program at step t, and whether that step
 * is in the phase's amber (R19); -1 if the junction has no phases */
static int fixed_phase(const Oracle* O, int j, long t, int* in_amber) {
    int p0 = O->junc_phase_off[j], P = O->junc_phase_off[j + 1] - p0;
    long cycle = 0;
    for (int p = 0; p < P; ++p) cycle += O->phase_green[p0 + p] + O->phase_amber[p0 + p];
    *in_amber = 0;
    if (P == 0 || cycle <= 0) return -1;
    long c = (t + O->junc_offset[j]) % cycle;
    if (c < 0) c += cycle;
    for (int p = 0; p < P; ++p) {
        long g = O->phase_green[p0 + p], a = O->phase_amber[p0 + p];
        if (c < g + a) {
            *in_amber = c >= g;
            return p;
        }
        c -= g + a;
    }
    return -1; /* not reached */
}

int mo_light(void* h, int jl, long t) {
    Oracle* O = (Oracle*)h;
    int j = O->jl_junction[jl];
    int mask = O->jl_mask[jl];
    int P = O->junc_phase_off[j + 1] - O->junc_phase_off[j];
    if (O->junc_policy[j] == POLICY_NONE) return LIGHT_GREEN;
    if (O->junc_policy[j] == POLICY_MANUAL)
        return ((mask >> O->junc_manual[j]) & 1) ? LIGHT_GREEN : LIGHT_RED;
    if (O->junc_policy[j] == POLICY_MAXP) {
        if (P == 0) return LIGHT_GREEN;
        int p = O->mp_phase[j], q = O->mp_pending[j];
        if (!((mask >> p) & 1)) return LIGHT_RED;
        if (q < 0) return LIGHT_GREEN;
        return ((mask >> q) & 1) ? LIGHT_GREEN : LIGHT_AMBER;
    }
    int amber;
    int p = fixed_phase(O, j, t, &amber);
    if (p < 0) return LIGHT_GREEN;
    if (!((mask >> p) & 1)) return LIGHT_RED;
    if (!amber) return LIGHT_GREEN;
    int nxt = (p + 1) % P;
    return ((mask >> nxt) & 1) ? LIGHT_GREEN : LIGHT_AMBER;
}

/* policy for n junctions; phases may be NULL unless policy == MANUAL.  A
 * junction switched to max pressure starts, green, the phase it shows at the
 * current step (R23). */
void mo_set_signal(void* h, int n, const int* junctions, int policy, const int* phases) {
    Oracle* O = (Oracle*)h;
    for (int k = 0; k < n; ++k) {
        int j = junctions[k];
        if (policy == POLICY_MAXP) {
            int shown = 0;
            if (O->junc_policy[j] == POLICY_FIXED) {
                int amber;
                int p = fixed_phase(O, j, O->step, &amber);
                shown = p < 0 ? 0 : p;
            } else if (O->junc_policy[j] == POLICY_MANUAL) {
                shown = O->junc_manual[j];
            } else if (O->junc_policy[j] == POLICY_MAXP) {
                shown = O->mp_phase[j];
            }
            O->mp_phase[j] = shown;
            O->mp_elapsed[j] = 1;
            O->mp_pending[j] = -1;
        }
        O->junc_policy[j] = policy;
        if (policy == POLICY_MANUAL) O->junc_manual[j] = phases[k];
    }
}

/* R25 setters, effective from the next step */
void mo_set_lane_max_speed(void* h, int n, const int* lanes, const double* vmax) {
    Oracle* O = (Oracle*)h;
    for (int k = 0; k < n; ++k) O->vmax[lanes[k]] = vmax[k];
}

void mo_set_lane_restriction(void* h, int n, const int* lanes, const int* flags) {
    Oracle* O = (Oracle*)h;
    for (int k = 0; k < n; ++k) O->restricted[lanes[k]] = flags[k] != 0;
}

/* R26: replace the route of vehicle vid by roads[0..n); returns 0, or -1 if
 * the vehicle has arrived, the route does not start with the vehicle's road,
 * or two consecutive roads are not joined by a junction lane. */
static int roads_joined(const Oracle* O, int a, int b) {
    for (int l = O->road_lane_off[a]; l < O->road_lane_off[a + 1]; ++l)
        for (int j = O->jl_off[l]; j < O->jl_off[l + 1]; ++j)
            if (O->lane_road[O->jl_target[j]] == b) return 1;
    return 0;
}

int mo_set_vehicle_route(void* h, int vid, int n, const int* roads) {
    Oracle* O = (Oracle*)h;
    if (vid < 0 || vid >= O->n_veh || n < 1 || O->status[vid] == ST_ARRIVED) return -1;
    for (int k = 0; k < n; ++k)
        if (roads[k] < 0 || roads[k] >= O->n_roads) return -1;
    int prev = -1;  /* on a junction lane: the road just left stays in front */
    if (O->status[vid] == ST_WAITING) {
        if (roads[0] != O->lane_road[O->start_lane[vid]]) return -1;
    } else if (O->lane[vid] < O->n_road_lanes) {
        if (roads[0] != O->lane_road[O->lane[vid]]) return -1;
    } else {
        int jl = O->lane[vid];
        if (roads[0] != O->lane_road[O->jl_target[jl]]) return -1;
        prev = O->lane_road[O->jl_from[jl]];
    }
    for (int k = 0; k + 1 < n; ++k)
        if (!roads_joined(O, roads[k], roads[k + 1])) return -1;
    long need = O->routes_used + n + 1;
    if (need > O->routes_cap) {
        long cap = O->routes_cap * 2 > need ? O->routes_cap * 2 : need;
        O->routes = (int*)realloc(O->routes, sizeof(int) * cap);
        O->routes_cap = cap;
    }
    int beg = (int)O->routes_used, len = 0;
    if (prev >= 0) O->routes[beg + len++] = prev;
    for (int k = 0; k < n; ++k) O->routes[beg + len++] = roads[k];
    O->routes_used += len;
    O->route_beg[vid] = beg;
    O->route_len[vid] = len;
    if (O->status[vid] == ST_ACTIVE) O->rc[vid] = 0;
    return 0;
}

/* R28: plan masks of the junction lanes (jl_plans[k] for junction lane
 * n_road_lanes + k) and the plans of n roads */
void mo_set_lane_plans(void* h, const int* jl_plans) {
    Oracle* O = (Oracle*)h;
    for (int l = O->n_road_lanes; l < O->n_lanes; ++l) O->jl_plans[l] = jl_plans[l - O->n_road_lanes];
}

void mo_set_road_plan(void* h, int n, const int* roads, const int* plans) {
    Oracle* O = (Oracle*)h;
    for (int k = 0; k < n; ++k) O->road_plan[roads[k]] = plans[k];
}

/* R24 metrics of the current state: queue length per lane (out[n_lanes]) and
 * average vehicle speed per road (out[n_roads]) */
void mo_lane_queue(void* h, int* out) {
    Oracle* O = (Oracle*)h;
    for (int l = 0; l < O->n_lanes; ++l) out[l] = 0;
    for (int i = 0; i < O->n_veh; ++i) {
        if (O->status[i] != ST_ACTIVE) continue;
        int l = O->lane[i];
        if (O->v[i] < 0.1 && O->L[l] - O->s[i] <= 50.0) out[l]++;
    }
}

void mo_road_speed(void* h, double* out) {
    Oracle* O = (Oracle*)h;
    double* sum = (double*)xcalloc(O->n_roads, sizeof(double));
    long* cnt = (long*)xcalloc(O->n_roads, sizeof(long));
    for (int i = 0; i < O->n_veh; ++i) {
        if (O->status[i] != ST_ACTIVE) continue;
        int r = O->lane_road[O->lane[i]];
        if (r < 0) continue;  /* junction lanes belong to no road */
        sum[r] += O->v[i];
        cnt[r]++;
    }
    for (int r = 0; r < O->n_roads; ++r) {
        if (cnt[r] > 0) {
            out[r] = sum[r] / (double)cnt[r];
        } else {
            double m = 0.0;
            int nl = O->road_lane_off[r + 1] - O->road_lane_off[r];
            for (int l = O->road_lane_off[r]; l < O->road_lane_off[r + 1]; ++l) m += O->vmax[l];
            out[r] = m / nl;
        }
    }
    free(sum); free(cnt);
}

/* max-pressure state of junction j: out = [phase, steps in the current green
 * or amber interval (counting the current step), phase after the amber or
 * -1 while green] */
void mo_signal_state(void* h, int j, int* out) {
    Oracle* O = (Oracle*)h;
    out[0] = O->mp_phase[j]; out[1] = O->mp_elapsed[j]; out[2] = O->mp_pending[j];
}

/* Advance every max-pressure junction from step t to t+1 using the lane
 * counts of the step-t snapshot (R23). */
static void maxp_advance(Oracle* O, const int* lane_cnt) {
    long* press = (long*)xcalloc((size_t)O->n_junctions * 8, sizeof(long));
    for (int jl = O->n_road_lanes; jl < O->n_lanes; ++jl) {
        int j = O->jl_junction[jl];
        if (O->junc_policy[j] != POLICY_MAXP || !jl_available(O, jl)) continue;
        long d = (long)lane_cnt[O->jl_from[jl]] - (long)lane_cnt[O->jl_target[jl]];
        for (int p = 0; p < 8; ++p)
            if ((O->jl_mask[jl] >> p) & 1) press[(size_t)j * 8 + p] += d;
    }
    for (int j = 0; j < O->n_junctions; ++j) {
        if (O->junc_policy[j] != POLICY_MAXP) continue;
        int p0 = O->junc_phase_off[j], P = O->junc_phase_off[j + 1] - p0;
        if (P == 0) continue;
        int p = O->mp_phase[j], q = O->mp_pending[j], e = O->mp_elapsed[j];
        if (q >= 0) {                               /* amber of p, towards q */
            if (e >= O->phase_amber[p0 + p]) { p = q; q = -1; e = 1; }
            else e += 1;
        } else if (e >= O->phase_green[p0 + p]) {  /* minimum green served */
            int best = p;
            for (int k = 0; k < P; ++k) {
                long pk = press[(size_t)j * 8 + k], pb = press[(size_t)j * 8 + best];
                if (pk > pb || (pk == pb && best != p && k < best)) best = k;
            }
            if (best != p) {
                if (O->phase_amber[p0 + p] > 0) { q = best; e = 1; }
                else { p = best; e = 1; }
            } else {
                e += 1;
            }
        } else {
            e += 1;
        }
        O->mp_phase[j] = p; O->mp_pending[j] = q; O->mp_elapsed[j] = e;
    }
    free(press);
}

/* ------------------------------------------------------------------------ */
/* IDM, App. B.3 equations (1)-(2); delta = 4 taken as ((v/v0)^2)^2 (R15).  */
static double idm_free(const Oracle* O, double v, double v0) {
    double r = v / v0, r2 = r * r;
    return O->a_max * (1.0 - r2 * r2);
}

static double idm(const Oracle* O, double v, double v0, double gap, double dv) {
    double r = v / v0, r2 = r * r;
    double dyn = v * O->T + v * dv / (2.0 * sqrt(O->a_max * O->b_comf));
    double sstar = O->s0 + (dyn > 0.0 ? dyn : 0.0);
    double g = gap > 1e-3 ? gap : 1e-3;
    double q = sstar / g;
    return O->a_max * (1.0 - r2 * r2 - q * q);
}

double mo_idm(void* h, double v, double v0, double gap, double dv) {
    return idm((Oracle*)h, v, v0, gap, dv);
}
double mo_idm_free(void* h, double v, double v0) { return idm_free((Oracle*)h, v, v0); }

/* p_LC, App. B.3 with reading R3 */
static double p_lc(const Oracle* O, double uT) {
    if (uT >= 1.0) return O->p_hi;
    if (uT > 0.0) return O->p_lo + (O->p_hi - O->p_lo) * uT;
    return O->p_lo;
}
double mo_p_lc(void* h, double uT) { return p_lc((Oracle*)h, uT); }

/* ------------------------------------------------------------------------ */
/* Sensing by linear scan (plain definition of the paper's index, R16).      */
static int ahead_of(const Snap* S, int x, double s_y, int y) {
    return S->s[x] > s_y || (S->s[x] == s_y && x < y);
}

/* nearest vehicle ahead of the point (s, id) on lane, excluding id */
static int leader_on(const Snap* S, int lane, double s, int id) {
    int best = -1;
    for (int k = 0; k < S->lane_cnt[lane]; ++k) {
        int m = S->members[S->lane_first[lane] + k];
        if (m == id || !ahead_of(S, m, s, id)) continue;
        if (best < 0 || ahead_of(S, best, S->s[m], m)) best = m;
    }
    return best;
}

/* nearest vehicle behind the point (s, id) on lane, excluding id */
static int follower_on(const Snap* S, int lane, double s, int id) {
    int best = -1;
    for (int k = 0; k < S->lane_cnt[lane]; ++k) {
        int m = S->members[S->lane_first[lane] + k];
        if (m == id || ahead_of(S, m, s, id)) continue;
        if (best < 0 || ahead_of(S, m, S->s[best], best)) best = m;
    }
    return best;
}

/* the rearmost vehicle of a lane (-1 if empty) */
static int rearmost_on(const Snap* S, int lane) {
    int best = -1;
    for (int k = 0; k < S->lane_cnt[lane]; ++k) {
        int m = S->members[S->lane_first[lane] + k];
        if (best < 0 || ahead_of(S, best, S->s[m], m)) best = m;
    }
    return best;
}

/* next lane on vehicle vid's route after `lane`, where the vehicle's route
 * cursor is rc (index of the road just left when on a junction lane).
 * Writes the cursor that applies on the returned lane.  -1 if none. */
static int next_lane(const Oracle* O, int vid, int lane, int rc, int* rc_next) {
    int r0 = O->route_beg[vid], last = O->route_len[vid] - 1;
    if (lane < O->n_road_lanes) {
        if (rc >= last) return -1;
        int out_road = O->routes[r0 + rc + 1];
        for (int j = O->jl_off[lane]; j < O->jl_off[lane + 1]; ++j)
            if (O->lane_road[O->jl_target[j]] == out_road && jl_available(O, j)) { *rc_next = rc; return j; }
        return -2; /* route not drivable from this lane */
    }
    *rc_next = rc + 1;
    return O->jl_target[lane];
}

/* acceleration of a follower f on lane fl towards leader ld (in-lane only;
 * used for the MOBIL politeness terms, reading R2) */
static double acc_pair(const Oracle* O, const Snap* S, int f, int fl, int ld, double s_ld,
                       double v_ld) {
    double v0 = O->v0f[f] * O->vmax[fl];
    if (ld < 0) return idm_free(O, S->v[f], v0);
    return idm(O, S->v[f], v0, s_ld - O->len - S->s[f], S->v[f] - v_ld);
}

typedef struct {
    double a;          /* acceleration on the lane */
    int has_leader;    /* a leader (own or lookahead) bounds the displacement */
    double gap;        /* its gap */
    int stop;          /* red/amber stop line active */
    double stop_gap;   /* L - s */
    int leader;        /* leader id or -1 */
    int overlap;       /* own-lane leader with negative gap */
} LaneAcc;

/* Ego acceleration when driving on `lane` at (s, v) with route cursor rc:
 * min over the leader (own lane, else lookahead R11) and the stop line (R12). */
static LaneAcc accel_on_lane(const Oracle* O, const Snap* S, int vid, int lane, double s,
                             double v, int rc) {
    LaneAcc r;
    memset(&r, 0, sizeof(r));
    r.leader = -1;
    double v0 = O->v0f[vid] * O->vmax[lane];
    double a = idm_free(O, v, v0);
    int ld = leader_on(S, lane, s, vid);
    int rc1 = rc;
    int nl1 = next_lane(O, vid, lane, rc, &rc1);
    if (ld >= 0) {
        double gap = S->s[ld] - O->len - s;
        a = idm(O, v, v0, gap, v - S->v[ld]);
        r.has_leader = 1; r.gap = gap; r.leader = ld;
        r.overlap = gap < 0.0;
    } else if (nl1 >= 0) {
        double base = O->L[lane] - s;
        int nl = nl1, rcn = rc1;
        for (int k = 0; k < 2 && nl >= 0; ++k) {
            int rr = rearmost_on(S, nl);
            if (rr >= 0) {
                double gap = base + S->s[rr] - O->len;
                a = idm(O, v, v0, gap, v - S->v[rr]);
                r.has_leader = 1; r.gap = gap; r.leader = rr;
                break;
            }
            base += O->L[nl];
            int rcm = rcn;
            nl = (k == 0) ? next_lane(O, vid, nl, rcn, &rcm) : -1;
            rcn = rcm;
        }
    }
    if ((lane < O->n_road_lanes && nl1 >= O->n_road_lanes && S->light[nl1] != LIGHT_GREEN) ||
        (nl1 >= 0 && O->restricted[nl1]) || (lane < O->n_road_lanes && nl1 == -2)) {
        double gs = O->L[lane] - s;
        double as = idm(O, v, v0, gs, v);
        if (as < a) a = as;
        r.stop = 1; r.stop_gap = gs;
    }
    r.a = a;
    return r;
}

/* Full per-vehicle decision (everything before conflict resolution). */
typedef struct {
    LaneAcc own;
    int eligible, attempted, mandatory, cand, dir, tl, TL, TF;
    double u, scale;
    LaneAcc tgt;          /* ego on the chosen target lane */
    int flag;
    /* diagnostics */
    double uL, uR, pLC, uT, u_att, u_lc, u_dir;
    int feasL, feasR;
    double at_ego[2], a_new[2], at_new[2], a_old, at_old;
    int TLs[2], TFs[2], OF, OL;
} Decision;

/* road lane l has a junction lane to road r (R27) */
static int has_access(const Oracle* O, int l, int r) {
    for (int j = O->jl_off[l]; j < O->jl_off[l + 1]; ++j)
        if (O->lane_road[O->jl_target[j]] == r && jl_available(O, j)) return 1;
    return 0;
}

static Decision decide(const Oracle* O, const Snap* S, int vid, long t) {
    Decision D;
    memset(&D, 0, sizeof(D));
    D.tl = D.TL = D.TF = -1;
    D.TLs[0] = D.TLs[1] = D.TFs[0] = D.TFs[1] = D.OF = D.OL = -1;
    int lane = S->lane[vid];
    double s = S->s[vid], v = S->v[vid];
    D.own = accel_on_lane(O, S, vid, lane, s, v, S->rc[vid]);
    if (lane >= O->n_road_lanes) return D;              /* no changes in junctions */
    int road = O->lane_road[lane];
    int lo = O->road_lane_off[road], hi = O->road_lane_off[road + 1];
    if (hi - lo < 2) return D;
    D.eligible = 1;
    /* the next road of the route and the lane group giving access to it (R27) */
    int rcv = S->rc[vid];
    int next_road = rcv < O->route_len[vid] - 1 ? O->routes[O->route_beg[vid] + rcv + 1] : -1;
    if (next_road >= 0 && !has_access(O, lane, next_road)) {
        /* mandatory change towards the nearest lane of the group */
        int best = -1;
        for (int k = lo; k < hi; ++k)
            if (has_access(O, k, next_road) && (best < 0 || abs(k - lane) < abs(best - lane))) best = k;
        D.mandatory = 1;
        if (best < 0) return D;
        int dir = best < lane ? -1 : +1, tl = lane + dir;
        if (O->restricted[tl]) return D;
        int TL = leader_on(S, tl, s, vid), TF = follower_on(S, tl, s, vid);
        double pos_scale = s > 1.0 ? s : 1.0;
        int ok = 1;
        if (TL >= 0) {
            double g = S->s[TL] - O->len - s;
            if (!(g > 0.0)) ok = 0;
            if (fabs(g) < O->band * pos_scale) D.flag = 1;
        }
        if (TF >= 0) {
            double g = s - O->len - S->s[TF];
            if (!(g > 0.0)) ok = 0;
            if (fabs(g) < O->band * pos_scale) D.flag = 1;
            double at_new = acc_pair(O, S, TF, tl, vid, s, v);
            if (!(at_new >= -O->b_safe)) ok = 0;
            double sc = fabs(at_new) > 1.0 ? fabs(at_new) : 1.0;
            if (fabs(at_new + O->b_safe) < O->band * sc) D.flag = 1;
        }
        if (!ok) return D;
        D.cand = 1; D.dir = dir; D.tl = tl; D.TL = TL; D.TF = TF;
        D.u = U_MAND; D.scale = 1.0;
        D.tgt = accel_on_lane(O, S, vid, tl, s, v, rcv);
        return D;
    }
    uint32_t ctr[4] = {(uint32_t)vid, (uint32_t)t, 0u, 0u}, w[4];
    mo_philox4x32_10(O->key0, O->key1, ctr, w);
    D.u_att = unit24(w[0]); D.u_lc = unit24(w[1]); D.u_dir = unit24(w[2]);
    if (!(D.u_att < O->p_att)) return D;
    D.attempted = 1;

    /* old follower and the ego's own-lane leader (for ã_old / a_old) */
    int OF = follower_on(S, lane, s, vid);
    int OL = leader_on(S, lane, s, vid);
    D.OF = OF; D.OL = OL;
    if (OF >= 0) {
        D.a_old = acc_pair(O, S, OF, lane, vid, s, v);
        D.at_old = OL >= 0 ? acc_pair(O, S, OF, lane, OL, S->s[OL], S->v[OL])
                           : acc_pair(O, S, OF, lane, -1, 0.0, 0.0);
    }
    double u[2] = {0, 0}, scl[2] = {0, 0};
    int feas[2] = {0, 0}, TLs[2] = {-1, -1}, TFs[2] = {-1, -1};
    LaneAcc tgt[2];
    memset(tgt, 0, sizeof(tgt));
    double pos_scale = s > 1.0 ? s : 1.0;
    for (int side = 0; side < 2; ++side) {         /* 0 = left (k-1), 1 = right (k+1) */
        int tl = side == 0 ? lane - 1 : lane + 1;
        if (tl < lo || tl >= hi || O->restricted[tl]) continue;
        if (next_road >= 0 && !has_access(O, tl, next_road)) continue;  /* leaves the group (R27) */
        int TL = leader_on(S, tl, s, vid), TF = follower_on(S, tl, s, vid);
        TLs[side] = TL; TFs[side] = TF;
        int ok = 1;
        if (TL >= 0) {
            double g = S->s[TL] - O->len - s;
            if (!(g > 0.0)) ok = 0;
            if (fabs(g) < O->band * pos_scale) D.flag = 1;
        }
        if (TF >= 0) {
            double g = s - O->len - S->s[TF];
            if (!(g > 0.0)) ok = 0;
            if (fabs(g) < O->band * pos_scale) D.flag = 1;
        }
        tgt[side] = accel_on_lane(O, S, vid, tl, s, v, S->rc[vid]);
        double at_ego = tgt[side].a;
        double a_new = 0, at_new = 0;
        if (TF >= 0) {
            a_new = TL >= 0 ? acc_pair(O, S, TF, tl, TL, S->s[TL], S->v[TL])
                            : acc_pair(O, S, TF, tl, -1, 0.0, 0.0);
            at_new = acc_pair(O, S, TF, tl, vid, s, v);
            if (!(at_new >= -O->b_safe)) ok = 0;
            double sc = fabs(at_new) > 1.0 ? fabs(at_new) : 1.0;
            if (fabs(at_new + O->b_safe) < O->band * sc) D.flag = 1;
        }
        u[side] = (at_ego - D.own.a) + O->pol * ((at_new - a_new) + (D.at_old - D.a_old)) - O->a_th;
        scl[side] = fabs(at_ego) + fabs(D.own.a) +
                    O->pol * (fabs(at_new) + fabs(a_new) + fabs(D.at_old) + fabs(D.a_old)) + O->a_th;
        feas[side] = ok;
        D.at_ego[side] = at_ego; D.a_new[side] = a_new; D.at_new[side] = at_new;
    }
    D.uL = u[0]; D.uR = u[1]; D.feasL = feas[0]; D.feasR = feas[1];
    for (int sd = 0; sd < 2; ++sd) { D.TLs[sd] = TLs[sd]; D.TFs[sd] = TFs[sd]; }
    /* magnitude of the terms that decide: feasible sides only (R22) */
    double scale = 1.0;
    for (int sd = 0; sd < 2; ++sd)
        if (feas[sd] && scl[sd] > scale) scale = scl[sd];
    D.scale = scale;
    double uLp = (feas[0] && u[0] > 0.0) ? u[0] : 0.0;
    double uRp = (feas[1] && u[1] > 0.0) ? u[1] : 0.0;
    double uT = uLp + uRp;
    D.uT = uT;
    D.pLC = p_lc(O, uT);
    /* p_LC depends on u_T only below 1; above it is the constant p_hi */
    double band_p = (uT < 1.0 + O->band * scale) ? O->band * scale : O->band;
    if (fabs(D.u_lc - D.pLC) < band_p) D.flag = 1;
    if (!(D.u_lc < D.pLC)) return D;
    int side = -1;
    if (uT > 0.0) {
        double q = uLp - D.u_dir * uT;
        if (fabs(q) < O->band * scale) D.flag = 1;
        if (uT < O->band * scale) D.flag = 1;
        side = q > 0.0 ? 0 : 1;
    } else {
        if (feas[0] && feas[1]) side = D.u_dir < 0.5 ? 0 : 1;
        else if (feas[0]) side = 0;
        else if (feas[1]) side = 1;
        if (side >= 0 && uT < O->band * scale) D.flag = 1;
    }
    if (side < 0) return D;
    D.cand = 1;
    D.dir = side == 0 ? -1 : +1;
    D.tl = side == 0 ? lane - 1 : lane + 1;
    D.TL = TLs[side]; D.TF = TFs[side];
    D.u = u[side];
    D.tgt = tgt[side];
    return D;
}

/* ------------------------------------------------------------------------ */
static void snap_build(const Oracle* O, Snap* S, long t) {
    int n = O->n_veh;
    S->n = n;
    S->active = (char*)xcalloc(n, 1);
    S->lane = (int*)xcalloc(n, sizeof(int));
    S->rc = (int*)xcalloc(n, sizeof(int));
    S->s = (double*)xcalloc(n, sizeof(double));
    S->v = (double*)xcalloc(n, sizeof(double));
    S->lane_cnt = (int*)xcalloc(O->n_lanes, sizeof(int));
    S->lane_first = (int*)xcalloc(O->n_lanes + 1, sizeof(int));
    S->members = (int*)xcalloc(n, sizeof(int));
    S->light = (int*)xcalloc(O->n_lanes, sizeof(int));
    for (int i = 0; i < n; ++i) {
        S->active[i] = O->status[i] == ST_ACTIVE;
        S->lane[i] = O->lane[i]; S->rc[i] = O->rc[i]; S->s[i] = O->s[i]; S->v[i] = O->v[i];
        if (S->active[i]) S->lane_cnt[S->lane[i]]++;
    }
    for (int l = 0; l < O->n_lanes; ++l) S->lane_first[l + 1] = S->lane_first[l] + S->lane_cnt[l];
    int* fill = (int*)xcalloc(O->n_lanes, sizeof(int));
    for (int i = 0; i < n; ++i)
        if (S->active[i]) { int l = S->lane[i]; S->members[S->lane_first[l] + fill[l]++] = i; }
    free(fill);
    for (int l = O->n_road_lanes; l < O->n_lanes; ++l) S->light[l] = mo_light((void*)O, l, t);
}

static void snap_free(Snap* S) {
    free(S->active); free(S->lane); free(S->rc); free(S->s); free(S->v);
    free(S->lane_cnt); free(S->lane_first); free(S->members); free(S->light);
}

/* does candidate x beat candidate y (R9) */
static int wins(const Decision* Dx, int x, const Decision* Dy, int y) {
    return Dx->u > Dy->u || (Dx->u == Dy->u && x < y);
}

static void step_once(Oracle* O) {
    const long t = O->step;
    const int n = O->n_veh;
    Snap S;
    snap_build(O, &S, t);
    Decision* D = (Decision*)xcalloc(n, sizeof(Decision));
    int* granted = (int*)xcalloc(n, sizeof(int));
    for (int k = 0; k < n; ++k) {
        int i = O->reverse_order ? n - 1 - k : k;
        O->flags[i] = 0;
        if (!S.active[i]) continue;
        D[i] = decide(O, &S, i, t);
        if (D[i].own.overlap) O->m_overlaps++;
        if (D[i].attempted) O->m_mobil++;
    }
    /* conflict resolution among candidates, bucketed by target lane (R9) */
    int* tcnt = (int*)xcalloc(O->n_lanes + 1, sizeof(int));
    for (int i = 0; i < n; ++i) if (S.active[i] && D[i].cand) tcnt[D[i].tl + 1]++;
    for (int l = 0; l < O->n_lanes; ++l) tcnt[l + 1] += tcnt[l];
    int* tlist = (int*)xcalloc(n, sizeof(int));
    int* tfill = (int*)xcalloc(O->n_lanes, sizeof(int));
    for (int i = 0; i < n; ++i)
        if (S.active[i] && D[i].cand) tlist[tcnt[D[i].tl] + tfill[D[i].tl]++] = i;
    for (int k = 0; k < n; ++k) {
        int i = O->reverse_order ? n - 1 - k : k;
        if (!S.active[i] || !D[i].cand) continue;
        int ok = 1;
        int tl = D[i].tl;
        for (int q = tcnt[tl]; q < tcnt[tl + 1]; ++q) {
            int j = tlist[q];
            if (j == i || D[j].dir == D[i].dir) continue;
            if (D[j].TL != D[i].TL || D[j].TF != D[i].TF) continue;
            double sc = D[i].scale > D[j].scale ? D[i].scale : D[j].scale;
            if (fabs(D[i].u - D[j].u) < O->band * sc) D[i].flag = 1;
            if (!wins(&D[i], i, &D[j], j)) ok = 0;
        }
        granted[i] = ok;
    }
    free(tcnt); free(tlist); free(tfill);

    /* integration, transfer and arrival (R12, R13, R17) */
    double* v_upd = (double*)xcalloc(n, sizeof(double));
    for (int k = 0; k < n; ++k) {
        int i = O->reverse_order ? n - 1 - k : k;
        if (!S.active[i]) continue;
        const Decision* d = &D[i];
        int fl = d->flag ? F_FLAGGED : 0;
        if (d->cand) fl |= F_CANDIDATE;
        const LaneAcc* la = &d->own;
        int lane = S.lane[i];
        if (d->cand && granted[i]) { la = &d->tgt; lane = d->tl; fl |= F_CHANGED; O->m_lane_changes++; }
        if (d->cand && !granted[i]) fl |= F_CONFLICT_LOST;
        double s = S.s[i], v = S.v[i], a = la->a, dt = O->dt;
        double v_new = v + a * dt, disp;
        if (v_new >= 0.0) {
            disp = v * dt + 0.5 * a * dt * dt;
        } else {
            disp = -v * v / (2.0 * a);
            v_new = 0.0;
        }
        if (la->has_leader) { double c = la->gap > 0.0 ? la->gap : 0.0; if (disp > c) disp = c; }
        if (la->stop) { double c = la->stop_gap > 0.0 ? la->stop_gap : 0.0; if (disp > c) disp = c; }
        double s_new = s + disp;
        /* a vehicle held by the stop line cannot leave its lane (R13) */
        if (la->stop && s_new > O->L[lane]) s_new = O->L[lane];
        int rc = S.rc[i];
        int last = O->route_len[i] - 1;
        int arrived = 0, iter = 0;
        for (;;) {
            double Ll = O->L[lane];
            double sc = Ll > 1.0 ? Ll : 1.0;
            if (la->stop && iter == 0) break;
            if (lane < O->n_road_lanes && rc == last) {
                if (fabs(s_new - Ll) < O->band * sc) fl |= F_FLAGGED;
                if (s_new >= Ll) arrived = 1;
                break;
            }
            if (fabs(s_new - Ll) < O->band * sc) fl |= F_FLAGGED;
            if (!(s_new > Ll)) break;
            if (++iter > 4) { O->m_errors++; s_new = Ll; break; }
            int rcn = rc;
            int nl = next_lane(O, i, lane, rc, &rcn);
            if (nl < 0) { O->m_errors++; s_new = Ll; break; }
            s_new -= Ll;
            lane = nl; rc = rcn;
            fl |= F_TRANSFER;
        }
        v_upd[i] = v_new;
        if (arrived) {
            O->status[i] = ST_ARRIVED;
            O->lane[i] = -1;
            O->s[i] = 0.0; O->v[i] = v_new; O->rc[i] = rc;
            fl |= F_ARRIVED;
        } else {
            O->lane[i] = lane; O->s[i] = s_new; O->v[i] = v_new; O->rc[i] = rc;
        }
        if (fl & F_FLAGGED) O->m_flagged++;
        O->flags[i] = fl;
    }

    /* per-step metric sums in vehicle-id order (independent of processing order) */
    for (int i = 0; i < n; ++i) {
        if (!S.active[i]) continue;
        O->m_updates++;
        O->m_speed_sum += v_upd[i];
        if (O->flags[i] & F_ARRIVED) {
            O->m_arrived++;
            O->m_tt_sum += (double)(t + 1) * O->dt - (double)O->dep[i] * O->dt;
        }
    }
    free(v_upd);

    /* departure insertion against the snapshot (R18) */
    for (int l = 0; l < O->n_road_lanes; ++l) {
        int h = O->q_head[l];
        if (h >= O->q_off[l + 1] || O->restricted[l]) continue;
        int vid = O->q_ids[h];
        if (O->dep[vid] > t || O->status[vid] != ST_WAITING) continue;
        int r = rearmost_on(&S, l);
        int ok = 1, fl = F_INSERTED;
        if (r >= 0) {
            double g = S.s[r] - O->len - O->s0;
            double sc = S.s[r] > 1.0 ? S.s[r] : 1.0;
            if (fabs(g) < O->band * sc) fl |= F_FLAGGED;
            ok = g >= 0.0;
        }
        if (!ok) continue;
        O->status[vid] = ST_ACTIVE;
        O->lane[vid] = l; O->s[vid] = 0.0; O->v[vid] = 0.0; O->rc[vid] = 0;
        O->flags[vid] = fl;
        if (fl & F_FLAGGED) O->m_flagged++;
        O->q_head[l] = h + 1;
        O->m_inserted++;
    }
    free(D); free(granted);
    maxp_advance(O, S.lane_cnt);
    snap_free(&S);
    O->step = t + 1;
}

void mo_step(void* h, int n) {
    for (int k = 0; k < n; ++k) step_once((Oracle*)h);
}

void mo_set_reverse_order(void* h, int rev) { ((Oracle*)h)->reverse_order = rev; }

/* metrics: [step, n_active, n_waiting, n_arrived, tt_sum, speed_sum, updates,
 *           lane_changes, flagged, overlaps, inserted, errors, mobil_evals] */
void mo_get_metrics(void* h, double* out) {
    Oracle* O = (Oracle*)h;
    long act = 0, wait = 0;
    for (int i = 0; i < O->n_veh; ++i) {
        act += O->status[i] == ST_ACTIVE;
        wait += O->status[i] == ST_WAITING;
    }
    out[0] = (double)O->step; out[1] = (double)act; out[2] = (double)wait;
    out[3] = (double)O->m_arrived; out[4] = O->m_tt_sum; out[5] = O->m_speed_sum;
    out[6] = (double)O->m_updates; out[7] = (double)O->m_lane_changes;
    out[8] = (double)O->m_flagged; out[9] = (double)O->m_overlaps;
    out[10] = (double)O->m_inserted; out[11] = (double)O->m_errors;
    out[12] = (double)O->m_mobil;
}

void mo_get_state(void* h, int* status, int* lane, double* s, double* v, int* rc, int* flags) {
    Oracle* O = (Oracle*)h;
    for (int i = 0; i < O->n_veh; ++i) {
        status[i] = O->status[i]; lane[i] = O->lane[i]; s[i] = O->s[i]; v[i] = O->v[i];
        rc[i] = O->rc[i]; flags[i] = O->flags[i];
    }
}

/* Overwrite the vehicle state.  Waiting vehicles must form a suffix of every
 * start lane's FIFO; the queue heads are recomputed.  Metrics are kept. */
int mo_set_state(void* h, const int* status, const int* lane, const double* s, const double* v,
                 const int* rc, long step) {
    Oracle* O = (Oracle*)h;
    for (int i = 0; i < O->n_veh; ++i) {
        O->status[i] = status[i]; O->lane[i] = status[i] == ST_ACTIVE ? lane[i] : -1;
        O->s[i] = s[i]; O->v[i] = v[i]; O->rc[i] = rc[i]; O->flags[i] = 0;
    }
    for (int l = 0; l < O->n_road_lanes; ++l) {
        int hh = O->q_off[l];
        while (hh < O->q_off[l + 1] && O->status[O->q_ids[hh]] != ST_WAITING) ++hh;
        for (int k = hh; k < O->q_off[l + 1]; ++k)
            if (O->status[O->q_ids[k]] != ST_WAITING) return -1;
        O->q_head[l] = hh;
    }
    O->step = step;
    return 0;
}

/* Diagnostics of vehicle vid's decision in the current state (no state
 * change): out = [a_own, eligible, attempted, cand, dir, u, uL, uR, feasL,
 * feasR, uT, pLC, u_att, u_lc, u_dir, at_ego_L, at_ego_R, a_new_L, a_new_R,
 * at_new_L, at_new_R, a_old, at_old, flag, TL, TF, own_has_leader, own_gap,
 * own_stop, tgt_a, own_leader, TL_left, TF_left, TL_right, TF_right, OL, OF] */
void mo_decision(void* h, int vid, double* out) {
    Oracle* O = (Oracle*)h;
    Snap S;
    snap_build(O, &S, O->step);
    Decision D;
    memset(&D, 0, sizeof(D));
    if (S.active[vid]) D = decide(O, &S, vid, O->step);
    if (!S.active[vid]) { D.own.leader = -1; D.TLs[0] = D.TLs[1] = D.TFs[0] = D.TFs[1] = -1; D.OL = D.OF = -1; D.TL = D.TF = -1; }
    double vals[37] = {D.own.a, D.eligible, D.attempted, D.cand, D.dir, D.u, D.uL, D.uR,
                       D.feasL, D.feasR, D.uT, D.pLC, D.u_att, D.u_lc, D.u_dir,
                       D.at_ego[0], D.at_ego[1], D.a_new[0], D.a_new[1], D.at_new[0],
                       D.at_new[1], D.a_old, D.at_old, D.flag, D.TL, D.TF,
                       D.own.has_leader, D.own.gap, D.own.stop, D.tgt.a, D.own.leader,
                       D.TLs[0], D.TFs[0], D.TLs[1], D.TFs[1], D.OL, D.OF};
    memcpy(out, vals, sizeof(vals));
    snap_free(&S);
}
