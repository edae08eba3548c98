/*
 * moss.h — C ABI of the GB300 (sm_103a) microscopic traffic-simulation step.
 *
 * The library advances city-scale road networks one discrete time step at a
 * time on one GPU, following the per-timestep vehicle update of arxiv
 * 2406.10661 ("A GPU-accelerated Large-scale Simulator for Transportation
 * System Optimization Benchmarking"):
 *   - two-phase step: every vehicle reads the previous step's snapshot and
 *     writes only its own next state (§3.1, "Two-phase Parallel Process");
 *   - sensing of the leader/follower on the own lane, the adjacent lanes and
 *     the next lane of the route (§3.1, "Vehicle Sensing Indexes"; App. B.3);
 *   - IDM car following (App. B.3, equations (1)-(2), delta = 4), randomized
 *     MOBIL lane changing (App. B.3) with deterministic conflict resolution;
 *   - red/amber stop before the next lane's signal (App. B.3), fixed-time,
 *     manual, no-signal and max-pressure policies (§3.2, "Traffic Signal");
 *   - lane groups with mandatory lane changes and road lane plans (App. B.3;
 *     §3.2, "Road"), lane speed limits and restrictions (§3.2, "Lane"),
 *     vehicle re-routing (§3.2, "Vehicle");
 *   - transfer across junctions, departure insertion and arrival handling
 *     (App. B.2, prepare/update streams);
 *   - throughput, average travelling time, network speed, lane queue length
 *     and road speed (§3.3).
 *
 * Units: metres, seconds, m/s.  One step advances dt seconds.  Vehicle state
 * is kept in FP32 (precision 32) or FP64 (precision 64, used to compare
 * trajectories with a double-precision reference).
 *
 * Conventions for all calls
 *   - Every call returns MOSS_OK (0) or a MOSS_E* code; nothing aborts or
 *     throws across the boundary.  moss_last_error() describes the last
 *     failure of a handle.
 *   - Input arrays are HOST memory owned by the caller; moss_create deep-copies
 *     them, so they may be freed after it returns.
 *   - A handle owns all device memory it allocates and releases it in
 *     moss_destroy.  Calls on one handle must not run concurrently.
 *   - Work is enqueued on the handle's CUDA stream (the caller's stream if one
 *     is given to moss_create, else a stream the handle creates).  moss_step
 *     is asynchronous; moss_get_metrics / moss_get_state / moss_synchronize
 *     wait for the stream and report device-side errors raised meanwhile
 *     (MOSS_ETIMEOUT for a bounded device wait that ran out, MOSS_EDEVICE for
 *     an inconsistency found on the device).
 */
#ifndef MOSS_H
#define MOSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MOSS_OK 0
#define MOSS_EINVAL 1   /* invalid argument or inconsistent input arrays */
#define MOSS_ENOMEM 2   /* device or host allocation failed */
#define MOSS_ECUDA 3    /* a CUDA runtime call failed */
#define MOSS_ETIMEOUT 4 /* a bounded device-side wait gave up */
#define MOSS_EBUDGET 5  /* the request does not fit the given memory budget */
#define MOSS_EDEVICE 6  /* the device reported an inconsistent state */

#define MOSS_POLICY_FIXED_TIME 0 /* the network's built-in phase program */
#define MOSS_POLICY_MANUAL 1     /* the phase set by moss_set_signal_phase */
#define MOSS_POLICY_NONE 2       /* no signal: every junction lane is green */
/* adaptive maximum pressure (§3.2): the pressure of a junction lane is the
 * number of vehicles on the road lane it leaves minus the number on the road
 * lane it feeds (this step's snapshot), the pressure of a phase the sum over
 * its green junction lanes; the junction holds its phase for the phase's
 * programmed green time, then takes the phase of maximal pressure (its
 * current phase when that one is maximal, else the smallest index) for the
 * next step, changing through the current phase's programmed amber.  Set on
 * a junction, it starts the phase the junction shows at that step, green. */
#define MOSS_POLICY_MAX_PRESSURE 3

#define MOSS_ST_WAITING 0 /* not yet departed (or waiting for a safe entrance) */
#define MOSS_ST_ACTIVE 1  /* on a lane */
#define MOSS_ST_ARRIVED 2 /* trip finished */

/* per-vehicle flags of the last step (MossState.flags) */
#define MOSS_F_FLAGGED 1       /* a decision quantity was within flag_band of its threshold */
#define MOSS_F_CHANGED 2       /* changed lane */
#define MOSS_F_CANDIDATE 4     /* decided to change lane (before conflict resolution) */
#define MOSS_F_TRANSFER 8      /* crossed the end of a lane */
#define MOSS_F_ARRIVED 16      /* finished its trip this step */
#define MOSS_F_INSERTED 32     /* departed this step */
#define MOSS_F_CONFLICT_LOST 64 /* lost a lane-change conflict */

/*
 * Road network (App. B.1: lanes, roads, junctions).  All arrays host memory.
 *   Lanes [0, n_road_lanes) are road lanes, grouped by road: road r owns lanes
 *   [road_lane_off[r], road_lane_off[r+1]), ordered from the leftmost (lane
 *   change "left" = index - 1) to the rightmost.  Lanes [n_road_lanes,
 *   n_lanes) are junction lanes, grouped by the road lane they leave:
 *   junction lanes leaving road lane l are [jl_off[l], jl_off[l+1]) (absolute
 *   lane ids, jl_off has n_road_lanes+1 entries, jl_off[0] = n_road_lanes,
 *   jl_off[n_road_lanes] = n_lanes).  For junction lane j (index
 *   j - n_road_lanes): jl_target = the road lane it feeds, jl_junction = its
 *   junction, jl_mask bit p = green in phase p (p < 8).
 *   Junction k: phases [junc_phase_off[k], junc_phase_off[k+1]) with green
 *   and amber durations in whole steps; the program starts shifted by
 *   junc_offset[k] steps.  A junction with no phases has no signal.
 */
typedef struct MossNetwork {
    int32_t n_roads, n_road_lanes, n_lanes, n_junctions;
    const int32_t* road_lane_off;  /* [n_roads+1] */
    const float* lane_length;      /* [n_lanes] m, > 0 */
    const float* lane_vmax;        /* [n_lanes] m/s, > 0 */
    const int32_t* jl_off;         /* [n_road_lanes+1] */
    const int32_t* jl_target;      /* [n_lanes-n_road_lanes] */
    const int32_t* jl_junction;    /* [n_lanes-n_road_lanes] */
    const int32_t* jl_mask;        /* [n_lanes-n_road_lanes] */
    const int32_t* junc_offset;    /* [n_junctions] steps */
    const int32_t* junc_phase_off; /* [n_junctions+1] */
    const int32_t* phase_green;    /* [junc_phase_off[n_junctions]] steps */
    const int32_t* phase_amber;    /* [junc_phase_off[n_junctions]] steps */
    /* lane function plans (§3.2 "Road"; optional, NULL = one plan): bit p of
     * jl_plans[j - n_road_lanes] = junction lane j exists in plan p (p < 8).
     * Every road starts in plan 0; moss_set_road_lane_plan switches it.  A
     * junction lane outside the current plan of its road gives no access to
     * its out-road (the lane-group rules apply) and carries no pressure. */
    const int32_t* jl_plans;       /* [n_lanes-n_road_lanes] or NULL */
} MossNetwork;

/*
 * Travel demand (§3.1 "Simulator Inputs"): vehicle i (id = i) drives the
 * road sequence routes[route_off[i] .. route_off[i+1]), consecutive roads
 * connected through a junction lane from at least one lane (a vehicle on a
 * lane without access to its next road stops at the lane end and changes
 * towards the lanes that have it: App. B.3 lane groups); it departs no earlier
 * than step dep[i] on lane start_lane[i] (a lane of its first road) and has
 * desired-speed factor v0f[i] (desired speed = v0f * lane speed limit).
 */
typedef struct MossVehicles {
    int32_t n;
    const int32_t* route_off;  /* [n+1] */
    const int32_t* routes;     /* [route_off[n]] road ids */
    const int32_t* start_lane; /* [n] */
    const int32_t* dep;        /* [n] step */
    const float* v0f;          /* [n] */
} MossVehicles;

/*
 * Model parameters.  IDM (App. B.3): a_max, b_comf (comfortable
 * deceleration), T (headway), s0 (minimum gap), delta (must be 4).
 * Randomized MOBIL (App. B.3): politeness p, threshold a_th, safe braking
 * b_safe, attempt probability p_attempt, p_LC levels p_hi (u_T >= 1) and p_lo
 * (u_T = 0), linear in between.  flag_band: relative band around decision
 * thresholds inside which a decision is flagged (MOSS_F_FLAGGED).
 * Random draws: Philox4x32-10 with key (seed low word, seed high word XOR
 * scenario) and counter (vehicle id, step, 0, 0).
 * precision: 32 (FP32 state) or 64 (FP64 state).
 */
typedef struct MossParams {
    double dt, a_max, b_comf, T, s0, delta, veh_len, politeness, a_th, b_safe, p_attempt,
        p_hi, p_lo, flag_band;
    uint64_t seed;
    uint32_t scenario;
    int32_t precision;
} MossParams;

/* Cumulative metrics (§3.3): throughput = n_arrived; ATT = tt_sum / n_arrived;
 * network speed = speed_sum / vehicle_updates (speed after each update).
 * mobil_evals: vehicle updates that evaluated the MOBIL utilities (the
 * attempt draw passed on an eligible road lane). */
typedef struct MossMetrics {
    int64_t step, n_active, n_waiting, n_arrived;
    double tt_sum, speed_sum;
    int64_t vehicle_updates, lane_changes, flagged, overlaps, inserted, errors, mobil_evals;
} MossMetrics;

/* Per-vehicle state by vehicle id (host arrays of MossVehicles.n entries,
 * owned by the caller).  rc = index within the route of the current road (on
 * a junction lane: of the road just left).  flags: MOSS_F_* of the last step
 * (ignored by moss_set_state). */
typedef struct MossState {
    int32_t* status;
    int32_t* lane;
    double* s;
    double* v;
    int32_t* rc;
    int32_t* flags;
} MossState;

typedef struct MossHandle* moss_t;

/* Build a simulation of one scenario at step 0 with every vehicle waiting
 * (§3.1 "Python API": the initialization functions; §3.1 "Simulator Inputs":
 * a road network and a travel demand).  cuda_stream: a cudaStream_t to run
 * on, or NULL for a handle-owned stream.  The handle's device memory comes
 * from cudaMalloc (see moss_batch_create_with_allocator for a caller's
 * allocator).  Errors: MOSS_EINVAL (inconsistent arrays, delta != 4,
 * precision not 32/64), MOSS_ENOMEM, MOSS_ECUDA.  On error *out is NULL. */
int moss_create(const MossNetwork* net, const MossVehicles* veh, const MossParams* prm,
                void* cuda_stream, moss_t* out);

/* Enqueue n >= 0 steps of dt seconds (§3.1 "Python API": next_step, the call
 * that advances the simulation; App. B.2: one step is the prepare and update
 * phases over every vehicle).  Asynchronous on the handle's stream; replays
 * a captured CUDA graph.  MOSS_EINVAL for n < 0; device errors are reported
 * by the next waiting call. */
int moss_step(moss_t h, int n);

/* Set the phase of n junctions (batch setter, §3.1 "_batch" API, §3.2
 * set_tl_phase) and switch them to MOSS_POLICY_MANUAL, effective from the
 * next step.  junction_ids and phase_idx are host arrays of n entries.
 * MOSS_EINVAL if an id or phase is out of range (nothing is changed). */
int moss_set_signal_phase(moss_t h, int n, const int32_t* junction_ids, const int32_t* phase_idx);

/* Set the signal policy of n junctions (§3.2 set_tl_policy). */
int moss_set_signal_policy(moss_t h, int n, const int32_t* junction_ids, int32_t policy);

/*
 * Lane setters (§3.2 "Lane": set_lane_max_speed, set_lane_restriction), for
 * the lanes of a single-scenario handle (scenario 0 of a batch), effective
 * from the next step.  lane_ids and the values are host arrays of n entries.
 *   - moss_set_lane_max_speed: new speed limits (m/s, > 0); desired speeds
 *     are v0f x limit.
 *   - moss_set_lane_restriction: flags != 0 restrict a lane from passing: it
 *     is not entered — a vehicle whose next lane is restricted stops at the
 *     end of its lane as before a red light, lane changes into it are not
 *     considered, and no departure is inserted onto it; vehicles already on
 *     it drive on.  0 lifts the restriction.
 * Both wait for the handle's stream; MOSS_EINVAL for an id out of range or a
 * limit that is not > 0 (nothing is changed).
 */
int moss_set_lane_max_speed(moss_t h, int n, const int32_t* lane_ids, const float* vmax);
int moss_set_lane_restriction(moss_t h, int n, const int32_t* lane_ids, const int32_t* flags);

/*
 * Re-routing (§3.2 "Vehicle", set_vehicle_route) of n vehicles of a
 * single-scenario handle (scenario 0 of a batch): vehicle vehicle_ids[k]
 * gets the route roads[route_off[k] .. route_off[k+1]) (host arrays; road
 * ids).  The new route starts with the road the vehicle is on (a waiting
 * vehicle: the road of its start lane; a vehicle on a junction lane: the
 * road it is entering), every turn of it must be available from some lane,
 * and the vehicle arrives at the end of its last road as every trip does
 * (no destination inside a road).  All requests are checked before any is
 * applied: MOSS_EINVAL (arrived vehicle, route not starting with the
 * vehicle's road, roads not joined, duplicate or out-of-range ids) changes
 * nothing.  Effective from the next step; waits for the handle's stream.
 */
int moss_set_vehicle_route(moss_t h, int n, const int32_t* vehicle_ids, const int32_t* route_off,
                           const int32_t* roads);

/*
 * Lane function plans (§3.2 "Road", set_road_lane_plan) of n roads of a
 * single-scenario handle (scenario 0 of a batch): road road_ids[k] uses plan
 * plan_idx[k] (0..7) from the next step.  The vehicles on those roads get
 * their next lane again (a lane that loses access to a vehicle's next road
 * puts it outside its lane group); vehicles on junction lanes drive on.
 * Host arrays; MOSS_EINVAL for ids out of range (nothing changed).  Waits
 * for the handle's stream.
 */
int moss_set_road_lane_plan(moss_t h, int n, const int32_t* road_ids, const int32_t* plan_idx);

/*
 * Lane and road metrics of the current state (§3.3 "Lane Queue Length",
 * "Road Traveling Time"), into caller-owned host arrays:
 *   - moss_get_lane_queue: queue[l] for every lane l of the scenario = the
 *     vehicles with v < 0.1 m/s within the last 50 m of the lane;
 *   - moss_get_road_speed: speed[r] for every road r = the mean speed of the
 *     vehicles on its lanes (m/s), or the mean speed limit of its lanes when
 *     the road is empty.
 * The batch forms take the scenario index (lane and road ids local to it).
 * They wait for the handle's stream.
 */
int moss_get_lane_queue(moss_t h, int32_t* queue);
int moss_get_road_speed(moss_t h, double* speed);
int moss_batch_get_lane_queue(moss_t h, int scenario, int32_t* queue);
int moss_batch_get_road_speed(moss_t h, int scenario, double* speed);

/*
 * Signal state of n junctions at the current step, into host arrays of n
 * entries owned by the caller: the phase shown (-1 when every lane is green:
 * no signal, or a junction without phases), the steps spent in the current
 * green or amber interval (max-pressure junctions, counting the current step;
 * 0 otherwise) and the phase that follows the current amber (-1 while
 * green).  Single-scenario handles only (MOSS_EINVAL for a batch).  Waits for
 * the handle's stream.
 */
int moss_get_signal_state(moss_t h, int n, const int32_t* junction_ids, int32_t* phase, int32_t* elapsed,
                          int32_t* next_phase);

/* Wait for the handle's stream and copy the cumulative metrics into the
 * caller's struct (§3.3: throughput, average travelling time, network
 * speed).  Returns a pending device error (MOSS_ETIMEOUT, MOSS_EDEVICE). */
int moss_get_metrics(moss_t h, MossMetrics* out);

/*
 * Metrics without waiting for the stream (§3.3 metrics, read while the next
 * steps run): moss_metrics_enqueue copies the cumulative metrics of
 * `scenario` (0 for a single-scenario handle) as they are after all work
 * enqueued so far into readback slot `slot` (0 <= slot < MOSS_METRIC_SLOTS,
 * pinned host memory owned by the handle) and returns at once;
 * moss_metrics_read waits for that copy only and converts it, so a caller
 * can enqueue step k + 1 before reading step k.  Enqueuing into a slot whose
 * copy was not read yet first waits for that copy.  MOSS_EINVAL for a slot
 * out of range or read without an enqueue; device errors raised by the work
 * before the copy are reported by the read.
 */
#define MOSS_METRIC_SLOTS 64
int moss_metrics_enqueue(moss_t h, int scenario, int slot);
int moss_metrics_read(moss_t h, int slot, MossMetrics* out);

/* Wait for the handle's stream and copy the per-vehicle state (by id) into
 * the caller's arrays (§3.1 "Python API": the getter functions, such as the
 * vehicles' speeds and positions).  Returns a pending device error. */
int moss_get_state(moss_t h, MossState* out);

/* Replace the per-vehicle state and set the step counter (no counterpart in
 * the paper: checkpoint/resume, used to start from a given state in tests,
 * measurement and serving); s and v are rounded to the handle's precision.
 * Waiting vehicles must form the tail of each start lane's departure queue
 * ordered by (dep, id); active vehicles must sit on a lane of their route's
 * road rc with 0 <= s <= length.  Metrics are kept.  MOSS_EINVAL if the
 * state is inconsistent (nothing is changed). */
int moss_set_state(moss_t h, const MossState* in, int64_t step);

/* Wait for all work enqueued on the handle and report a pending device error
 * (no counterpart in the paper: the CUDA stream of the C ABI). */
int moss_synchronize(moss_t h);

/* Device bytes held by the handle (no counterpart in the paper; used for
 * admission by memory budget when serving). */
int moss_device_bytes(moss_t h, size_t* out);

/* Release the handle and its device memory (NULL is ignored); waits for the
 * handle's stream first.  No counterpart in the paper (resource management
 * of the C ABI). */
void moss_destroy(moss_t h);

/* Text of the handle's last error ("" if none); valid until the next call.
 * No counterpart in the paper (error reporting of the C ABI). */
const char* moss_last_error(moss_t h);

/*
 * Batching (no counterpart in the paper, whose "_batch" setters of §3.1
 * batch the calls of one simulation; this runs the many rollouts that the
 * optimisation loops of §4 need): n independent scenarios advanced
 * together, one launch per step kernel for all of them (scenarios of uneven
 * size share every launch).
 * Each scenario keeps its own vehicle ids, random streams (seed, scenario)
 * and step counter, so its trajectory is the same alone and in the batch.
 * Model parameters other than seed/scenario must be equal across scenarios
 * (MOSS_EINVAL otherwise).  moss_step, moss_synchronize, moss_device_bytes
 * and moss_destroy accept batch handles; per-scenario calls below take the
 * scenario index in [0, n).
 */
int moss_batch_create(int n, const MossNetwork* nets, const MossVehicles* vehs,
                      const MossParams* prms, void* cuda_stream, moss_t* out);

/*
 * Device allocator of a handle (no counterpart in the paper): lets a caller
 * whose framework owns the device memory — PyTorch's caching allocator, for
 * one — back every device buffer of a handle.  alloc returns device memory of
 * at least `bytes` bytes, aligned to 256 bytes, usable on cuda_stream (the
 * handle's stream), or NULL on failure (the call then returns MOSS_ENOMEM);
 * release gets back each pointer with its size and the same stream, after
 * the stream has finished with it.  ctx is passed through.  Both must be set.
 */
typedef struct MossAllocator {
    void* (*alloc)(size_t bytes, void* cuda_stream, void* ctx);
    void (*release)(void* ptr, size_t bytes, void* cuda_stream, void* ctx);
    void* ctx;
} MossAllocator;

/* moss_batch_create whose device buffers come from `allocator` (NULL: the
 * same as moss_batch_create).  The allocator must outlive the handle; setter
 * scratch and a growing route buffer are taken from it too.  MOSS_EINVAL if
 * only one of its functions is set. */
int moss_batch_create_with_allocator(int n, const MossNetwork* nets, const MossVehicles* vehs,
                                     const MossParams* prms, void* cuda_stream, const MossAllocator* allocator,
                                     moss_t* out);
int moss_batch_size(moss_t h, int* out);
int moss_batch_get_metrics(moss_t h, int scenario, MossMetrics* out);
int moss_batch_get_state(moss_t h, int scenario, MossState* out);
int moss_batch_set_signal_phase(moss_t h, int scenario, int n, const int32_t* junction_ids,
                                const int32_t* phase_idx);
/* The same for junctions of several scenarios in one call (§3.1 "_batch"
 * setters: one transfer for many calls): entry k sets junction
 * junction_ids[k] of scenario scenarios[k] (its own ids) to phase
 * phase_idx[k].  MOSS_EINVAL if any entry is out of range (nothing is
 * changed). */
int moss_batch_set_signal_phases(moss_t h, int n, const int32_t* scenarios, const int32_t* junction_ids,
                                 const int32_t* phase_idx);

/*
 * Slot batches: continuous batching for serving rollouts (no counterpart in
 * the paper; it serves the many concurrent rollouts of the optimisation
 * loops of §4).  A slot batch is one resident batch of n slots, each with a
 * fixed capacity; scenarios are loaded into free slots while the others
 * run, so one set of launches per step (moss_step) advances every scenario
 * in flight.  An empty, retired or frozen slot does not advance.
 *
 * Capacities: a slot takes any scenario with at most n_lanes lanes (road
 * and junction lanes), n_roads roads, n_junctions junctions, n_phases signal
 * phases in all, n_vehicles vehicles and n_route_entries route entries, and
 * without lane groups or lane plans.  The slot also holds one padding lane,
 * road and junction (isolated, empty) of its own.
 *
 * Per-slot calls take the slot index as the scenario index of the batch
 * calls (moss_batch_get_metrics, moss_batch_get_state,
 * moss_batch_set_signal_phase, moss_batch_get_lane_queue,
 * moss_batch_get_road_speed: with the loaded scenario's own ids and sizes).
 * Lane setters, re-routing, lane plans, signal policies and moss_set_state
 * are not available on slot batches (MOSS_EINVAL).
 */
typedef struct MossSlotCaps {
    int32_t n_lanes, n_roads, n_junctions, n_phases, n_vehicles, n_route_entries;
} MossSlotCaps;

/* Create a slot batch of n empty slots with the given capacities; prm gives
 * the model parameters every loaded scenario must share (seed and scenario
 * id may differ).  allocator: as for moss_batch_create_with_allocator (NULL:
 * cudaMalloc).  Errors: MOSS_EINVAL, MOSS_ENOMEM, MOSS_ECUDA. */
int moss_slots_create(int n, const MossSlotCaps* caps, const MossParams* prm, void* cuda_stream,
                      const MossAllocator* allocator, moss_t* out);

/* Load a scenario into slot `slot` at its step 0 (every vehicle waiting,
 * fixed-time signals, metrics zero, random streams from its own seed and
 * scenario id), to run from the next step.  The slot must be empty, or
 * retired with at least one moss_step enqueued since (that step removes its
 * vehicles).  The tables are copied in stream order behind the work already
 * enqueued, without waiting for it (the host arrays may be freed on return).
 * MOSS_EINVAL if the scenario is inconsistent, larger than the slot, has
 * lane groups or plans, or differs in model parameters; the slot is then
 * left empty. */
int moss_slot_load(moss_t h, int slot, const MossNetwork* net, const MossVehicles* veh, const MossParams* prm);

/* Retire slot `slot`: the next step removes its vehicles and the slot stops
 * advancing; enqueue or read its metrics first.  A slot that is empty or
 * retired already is left as it is.  Asynchronous (stream order). */
int moss_slot_retire(moss_t h, int slot);

/* Freeze slot `slot` once its own step counter reaches stop_at (its
 * vehicles, clock, signals and metrics stand still from then on; -1: never),
 * so that its results at that step can be read while other slots run on.
 * Asynchronous (stream order).  MOSS_EINVAL for a slot not loaded. */
int moss_slot_set_horizon(moss_t h, int slot, int64_t stop_at);

/*
 * Kernel timing for measurement: when enabled, every step records CUDA
 * events around each kernel on the handle's stream (graphs are not used
 * while enabled).  moss_kernel_times returns the summed milliseconds per
 * kernel since enabling, in the order (decide, lanescan, place, resolve) —
 * the launch order is decide, resolve, lanescan, place; resolve finishes the
 * lane-change candidates — and the number of timed steps.
 */
int moss_set_kernel_timing(moss_t h, int enable);
int moss_kernel_times(moss_t h, double* ms4, int64_t* steps);

/*
 * Launch form of a step (no counterpart in the paper, whose step is a
 * sequence of kernels on several streams, App. B.2): mode 0 (the default)
 * replays three kernels per step from a captured CUDA graph; mode 1 runs the
 * whole step as one cooperative launch (every block resident at once, the
 * kernels' work as phases separated by grid-wide barriers whose waits are
 * bounded: MOSS_ETIMEOUT), also graph-replayed.  Results do not depend on
 * the mode.  Waits for the handle's stream and re-captures the graphs.
 * MOSS_EINVAL for another mode, or mode 1 on a device without cooperative
 * launch.
 */
int moss_set_step_mode(moss_t h, int mode);

/* Kernel launches of the library per step in the current mode (3 in mode 0:
 * decide, lane scan with the conflict resolution, place; 1 in mode 1). */
int moss_step_launches(moss_t h, int* out);

/*
 * Autotuner of the launch schedule (no counterpart in the paper): times the
 * next steps of the simulation (16 x trial_steps of them, 14 without
 * cooperative launch; they are simulated normally, and the results do not
 * depend on the schedule) under candidate schedules, keeps the fastest by
 * coordinate search over, in this order: k_decide blocks per SM {3,4,5}; the
 * weight of a road-lane vehicle in the split of the snapshot into k_decide's
 * block runs {0,1,2} (a junction-lane vehicle weighs 1; 0: the weight fitted each step); k_lanescan blocks
 * per SM {1,2,4}; lanes per thread of a lane-scan tile {16,8}; k_place
 * blocks per SM {4,8,16}; the step mode {0,1} (moss_set_step_mode).  Then it
 * re-captures the step graphs.  chosen3 (may be NULL) receives the chosen
 * decide/lanescan/place blocks per SM; moss_get_schedule returns the whole schedule.
 */
int moss_autotune(moss_t h, int trial_steps, int* chosen3);

/*
 * The launch schedule (no counterpart in the paper): out7 / in7 = k_decide,
 * k_lanescan and k_place blocks per SM, the road-lane weight of k_decide's
 * runs (0: fitted each step from the previous step's run times, the
 * default; 1..8: fixed), lanes per thread of a lane-scan tile (8 or 16), the step mode (0 or
 * 1), as moss_autotune describes, and the number of lane-change candidates
 * a k_decide block resolves itself at the end of its run (0..256, default
 * 256; the others are resolved by the first tickets of k_lanescan).
 * moss_set_schedule checks the ranges (blocks per SM 1..16 for k_decide,
 * 1..32 for the others; weight 0..8), waits for the handle's stream and
 * re-captures the step graphs; on an error the previous schedule stays.
 * Results never depend on the schedule.
 */
int moss_get_schedule(moss_t h, int* out7);
int moss_set_schedule(moss_t h, const int* in7);

/*
 * Failure-detection self-test (no counterpart in the paper).  Launches one
 * warp that runs the step's look-back wait (the decoupled scan of the lane
 * offsets) against a tile word that nothing ever publishes, so the bounded
 * wait must give up after its iteration limit (about a second) instead of
 * hanging.  Uses a 64-byte device buffer it allocates and frees itself, on
 * cuda_stream (NULL = legacy default stream), and waits for the stream.
 * Returns MOSS_ETIMEOUT when the wait gave up and the kernel reported it
 * (the expected result; the CUDA context stays usable), MOSS_EDEVICE if the
 * wait returned without reporting, MOSS_ECUDA if a CUDA call failed.
 */
int moss_selftest_bounded_wait(void* cuda_stream);

/*
 * Lane offsets without allocating (no counterpart in the paper: an addition
 * for callers that cannot call cudaMalloc, such as code running inside a
 * framework whose caching allocator owns the device memory, or a process
 * with a fixed memory reservation).
 *
 * Computes, for n_lanes lanes, the lane segments of the next snapshot from
 * the current ones: newsize(l) = d_off_cur[l+1] - d_off_cur[l] - d_leave[l] +
 * d_enter[l]; d_off_next[0..n_lanes] = exclusive prefix sums of newsize (the
 * last entry is the total); d_lbefore[0..n_lanes-1] = exclusive prefix sums
 * of d_leave.  Preconditions: every newsize(l) >= 0 (a lane cannot lose more
 * vehicles than it holds plus those entering), and the sums of newsize and of
 * d_leave over all lanes are below 2^31.  A negative newsize is reported
 * (d_off_next[n_lanes] = -1, the other entries are then meaningless); totals
 * of 2^31 or more are not detected.  All five arrays are DEVICE int32 arrays owned by the caller
 * (d_off_cur and d_off_next have n_lanes+1 entries).  The work is enqueued
 * on cuda_stream (NULL = the legacy default stream) and the call returns
 * without waiting.
 *
 * It allocates nothing: the scan's look-back words live in one file-scope
 * static device array of 32 KiB (plus 256 bytes), held by every GPU that
 * loads the library until the process exits.  Limit: n_lanes <=
 * MOSS_NOALLOC_MAX_LANES; larger sizes return MOSS_EINVAL.  The first call on
 * a device looks up that array's device address (and the SM count) with the
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture, and do not use the call across a
 * cudaDeviceReset (or a release of the device's primary context), after
 * which the kept address may no longer be the array's.  Every
 * call reuses the same array (each call clears it first), so calls that can
 * overlap on the GPU — on different streams, or from different threads —
 * race and must be serialised by the caller.  If a bounded device-side wait
 * gives up, d_off_next[n_lanes] is set to -1 as well.  Returns MOSS_OK, MOSS_EINVAL
 * (bad size or null array) or MOSS_ECUDA (a CUDA call failed).
 */
#define MOSS_NOALLOC_MAX_LANES (1 << 22)
int moss_lane_offsets_noalloc(int32_t n_lanes, const int32_t* d_off_cur, const int32_t* d_leave,
                              const int32_t* d_enter, int32_t* d_off_next, int32_t* d_lbefore,
                              void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MOSS_H */
