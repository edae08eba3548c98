// Kernels of one simulation step (see moss_device.cuh for the layout).
#pragma once

#include "moss_device.cuh"

namespace moss {

// entrant list of a lane for this step's tag (-1 if empty or stale)
__device__ __forceinline__ int list_head(const unsigned long long* head, int lane, int tag) {
    const unsigned long long h = head[lane];
    return (int)(h >> 32) == tag ? (int)(unsigned)(h & 0xffffffffull) : -1;
}

// append entrant q to the list of `lane`
__device__ __forceinline__ void list_push(unsigned long long* head, int32_t* enext, int lane, int q, int tag) {
    const unsigned long long prev =
        atomicExch(&head[lane], ((unsigned long long)(unsigned)tag << 32) | (unsigned)q);
    enext[q] = (int)(prev >> 32) == tag ? (int)(unsigned)(prev & 0xffffffffull) : -1;
}

// ---------------------------------------------------------------------------
// Departure insertion (R18) for start lane l: the head of its FIFO enters at
// s = 0, v = 0 when due and the snapshot's rearmost vehicle on the lane has
// s - len >= s0 (or the lane is empty).
template <typename Real>
__device__ void insert_departure(const Ctx<Real>& c, int l, int tag) {
    const int h = c.q_head[l];
    if (h >= c.q_off[l + 1]) return;
    const int vid = c.q_ids[h];
    const int sc = c.lane[l].scen;
    const long long t = c.scen_step[sc];
    if ((long long)c.dep[vid] > t) return;
    const int b = c.cur.off[l], e = c.cur.off[l + 1];
    int fl = F_INSERTED;
    if (e > b) {
        const Real sr = c.cur.a[e - 1].s;
        const Real g = sr - c.len - c.s0;
        const Real scl = sr > Real(1) ? sr : Real(1);
        if (rabs(g) < c.band * scl) fl |= F_FLAGGED;
        if (!(g >= Real(0))) return;
    }
    const int q = atomicAdd(&c.cnt->n_ent, 1);
    const int r0 = c.route_off[vid], r1 = c.route_off[vid + 1] - 1;
    int nl = -1;
    if (r0 < r1) {
        nl = jl_toward(c, c.lane[l], c.routes[r0 + 1]);
        if (nl < 0) atomicOr(&c.cnt->err, ERR_ROUTE);
    }
    RecA<Real> A;
    A.s = Real(0); A.v = Real(0); A.id = vid; A.lane = l;
    RecB B;
    B.v0f = c.v0f[vid]; B.rptr = r0; B.rlast = r1; B.nl = nl;
    c.ea[q] = A;
    c.eb[q] = B;
    atomicAdd(&c.enter[l], 1);
    list_push(c.head, c.enext, l, q, tag);
    c.q_head[l] = h + 1;
    c.vstatus[vid] = 1;
    c.vflags[vid] = int((t & 0xFFFFFF) << 8) | fl;
    long long* M = c.metrics + (long long)sc * M_NFIELDS;
    atomicAdd((unsigned long long*)&M[M_INSERTED], 1ull);
    atomicAdd((unsigned long long*)&M[M_CUR_ACTIVE], 1ull);
    if (fl & F_FLAGGED) atomicAdd((unsigned long long*)&M[M_FLAGGED], 1ull);
}

// ---------------------------------------------------------------------------
// Ballistic update with clamps (R12, R13), transfer and arrival (R17), and the
// outputs of one vehicle (slot i) driving on lane `nlane` (record ni) with
// lane kinematics la.  Returns 1 if the vehicle leaves its lane's segment.
template <typename Real>
__device__ __forceinline__ int integrate_emit(const Ctx<Real>& c, MetricAcc& acc, int i, const RecA<Real>& E,
                                              const RecB& EB, const LaneAcc<Real>& la, int nlane, int fl,
                                              bool own_overlap, long long t, int sc, int tag) {
    const int lane = E.lane;
    const Real s = E.s, v = E.v, a = la.a, dt = c.dt;
    Real vn = v + a * dt, disp;
    if (vn >= Real(0)) {
        disp = v * dt + Real(0.5) * a * dt * dt;
    } else {
        disp = -v * v / (Real(2) * a);
        vn = Real(0);
    }
    if (la.has_leader) { const Real cl = la.gap > Real(0) ? la.gap : Real(0); if (disp > cl) disp = cl; }
    if (la.stop) { const Real cl = la.stop_gap > Real(0) ? la.stop_gap : Real(0); if (disp > cl) disp = cl; }
    LaneInfo ni = c.lane[nlane];
    Real sn = s + disp;
    if (la.stop && sn > Real(ni.L)) sn = Real(ni.L);
    // The overshoot past the lane end is taken as disp - (L - s): L - s is
    // exact for s >= L/2 (Sterbenz), so the position on the next lane does
    // not lose the bits of L.
    int rptr = EB.rptr;
    const int rlast = EB.rlast;
    int nl = la.nl;
    bool arrived = false;
    Real ex = disp - (Real(ni.L) - s);  // distance beyond the end of nlane
    if (!la.stop) {
        for (int iter = 0;;) {
            const Real Ll = Real(ni.L);
            const Real scl = Ll > Real(1) ? Ll : Real(1);
            const bool road = ni.lo >= 0;
            if (rabs(ex) < c.band * scl) fl |= F_FLAGGED;
            if (road && rptr == rlast) {
                if (ex >= Real(0)) arrived = true;
                break;
            }
            if (!(ex > Real(0))) break;
            if (++iter > 4 || nl < 0) { atomicOr(&c.cnt->err, ERR_TRANSFER); sn = Ll; break; }
            sn = ex;
            fl |= F_TRANSFER;
            nlane = nl;
            ni = c.lane[nlane];
            if (road) {
                nl = ni.hi;  // entered a junction lane: next is its target road lane
            } else {
                rptr += 1;  // entered the next road
                nl = (rptr < rlast) ? jl_toward(c, ni, c.routes[rptr + 1]) : -1;
                if (rptr < rlast && nl < 0) atomicOr(&c.cnt->err, ERR_ROUTE);
            }
            ex = sn - Real(ni.L);
        }
    }
    if (arrived) fl |= F_ARRIVED;
    acc.m[0] += 1;
    acc.m[3] += speed_fixed(vn);
    if (fl & F_FLAGGED) acc.m[5] += 1;
    if (fl & F_CHANGED) acc.m[4] += 1;
    if (own_overlap) acc.m[6] += 1;
    if (fl) c.vflags[E.id] = int((t & 0xFFFFFF) << 8) | fl;
    if (arrived) {
        c.code[i] = C_ARRIVE;
        c.vstatus[E.id] = 2;
        acc.m[1] += 1;
        acc.m[2] += (t + 1) - (long long)c.dep[E.id];
        atomicAdd(&c.leave[lane], 1);
        long long* M = c.metrics + (long long)sc * M_NFIELDS;
        atomicAdd((unsigned long long*)&M[M_CUR_ACTIVE], (unsigned long long)(-1ll));
        atomicAdd((unsigned long long*)&M[M_CUR_ARRIVED], 1ull);
        return 1;
    }
    if (nlane == lane) {
        c.code[i] = C_STAY;
        SV<Real> w;
        w.s = sn; w.v = vn;
        c.stay[i] = w;
        return 0;
    }
    c.code[i] = C_MOVE;
    atomicAdd(&c.leave[lane], 1);
    const int q = atomicAdd(&c.cnt->n_ent, 1);
    RecA<Real> A;
    A.s = sn; A.v = vn; A.id = E.id; A.lane = nlane;
    RecB B;
    B.v0f = EB.v0f; B.rptr = rptr; B.rlast = rlast; B.nl = nl;
    c.ea[q] = A;
    c.eb[q] = B;
    atomicAdd(&c.enter[nlane], 1);
    list_push(c.head, c.enext, nlane, q, tag);
    return 1;
}

// ---------------------------------------------------------------------------
// k_decide: blocks [0, n_work) take 256-slot tiles of the current snapshot
// (one vehicle per thread); blocks [n_work, gridDim) run the insertion.
// MOSS_DECIDE_MIN_BLOCKS: resident blocks per SM the register budget targets.
#ifndef MOSS_DECIDE_MIN_BLOCKS
#define MOSS_DECIDE_MIN_BLOCKS 4
#endif
template <typename Real>
__global__ void __launch_bounds__(TILE, MOSS_DECIDE_MIN_BLOCKS) k_decide(Ctx<Real> c, int n_work) {
    if (c.cnt->err & ERR_POISON) return;
    const int tag = c.cnt->tag;
    if ((int)blockIdx.x >= n_work) {
        const int stride = (gridDim.x - n_work) * TILE;
        for (int k = (blockIdx.x - n_work) * TILE + threadIdx.x; k < c.n_start; k += stride)
            insert_departure(c, c.start_lanes[k], tag);
        return;
    }
    const int n = c.cnt->n_cur;
    const int n_tiles = (n + TILE - 1) / TILE;
    // each block takes a contiguous run of tiles: a thread's scenario (and so
    // its metric partials) changes rarely, and neighbouring lanes stay close
    const int per = (n_tiles + n_work - 1) / n_work;
    const int t_beg = blockIdx.x * per, t_end = min(n_tiles, t_beg + per);
    MetricAcc acc;
    macc_reset(acc, -1);
    for (int tile = t_beg; tile < t_end; ++tile) {
        const int i = tile * TILE + threadIdx.x;
        int leaver = 0;
        if (i < n) {
            const RecA<Real> E = c.cur.a[i];
            const int lane = E.lane;
            if ((unsigned)lane >= (unsigned)c.n_lanes) {
                atomicOr(&c.cnt->err, ERR_RANGE);
            } else {
                const int sc = c.lane[lane].scen;
                if (sc != acc.scen) {
                    macc_flush_thread(acc, c.metrics);
                    macc_reset(acc, sc);
                }
                const long long t = c.scen_step[sc];
                const uint32_t k0 = c.key0[sc], k1 = c.key1[sc];
                const int vbase = c.veh_base[sc];
                // job 0 is this vehicle; jobs 1.. are the rivals of a lane-change
                // candidate (R9): vehicles of the lane beyond the target lane that
                // fall into the same target-lane gap.  One call site of decide()
                // makes every recomputation bit-identical to the rival's own.
                Decision<Real> D;
                int fl = 0;
                bool granted = false;
                int r = 0, rend = 0;
                for (int job = 0;; ++job) {
                    const int slot = job == 0 ? i : r;
                    const Decision<Real> X = decide(c, slot, t, k0, k1, vbase);
                    if (job == 0) {
                        D = X;
                        fl = D.flag ? F_FLAGGED : 0;
                        if (!D.cand) break;
                        fl |= F_CANDIDATE;
                        granted = true;
                        const LaneInfo li = c.lane[lane];
                        const int ol = D.tl + D.dir;
                        if (ol < li.lo || ol >= li.hi) break;
                        const int ob = c.cur.off[ol], oe = c.cur.off[ol + 1];
                        r = ob; rend = oe;
                        if (D.TL >= 0) {
                            const RecA<Real> T = c.cur.a[D.TL];
                            r = partition_point(c, ob, oe, T.s, T.id);
                        }
                        if (D.TF >= 0) {
                            const RecA<Real> T = c.cur.a[D.TF];
                            rend = partition_point(c, ob, oe, T.s, T.id);
                        }
                        if (r >= rend) break;
                    } else {
                        if (X.cand && X.tl == D.tl) {
                            const Real sc2 = D.scale > X.scale ? D.scale : X.scale;
                            if (rabs(D.u - X.u) < c.band * sc2) fl |= F_FLAGGED;
                            const int rid = c.cur.a[r].id;
                            if (!(D.u > X.u || (D.u == X.u && E.id < rid))) granted = false;
                        }
                        if (++r >= rend) break;
                    }
                }
                if (D.att) acc.m[8] += 1;
                if (D.cand && !granted) fl |= F_CONFLICT_LOST;
                // a granted change drives on the target lane (its kinematics
                // recomputed from the same inputs)
                const RecB EB = c.cur.b[i];
                LaneAcc<Real> la = D.own;
                int nlane = lane;
                if (granted) {
                    fl |= F_CHANGED;
                    nlane = D.tl;
                    const LaneInfo ti = c.lane[nlane];
                    la = accel_on_lane(c, ti, E.s, E.v, Real(EB.v0f) * Real(ti.vmax), D.TL, D.nlt, EB.rptr,
                                       EB.rlast);
                }
                leaver = integrate_emit(c, acc, i, E, EB, la, nlane, fl, D.own.overlap != 0, t, sc, tag);
            }
        }
        // leavers of this tile (k_lanescan zeroes the counters after reading them)
        const unsigned lb = __ballot_sync(0xffffffffu, leaver);
        if ((threadIdx.x & 31) == 0 && lb) atomicAdd(&c.tile_leave[tile], __popc(lb));
    }
    macc_flush_block<TILE>(acc, c.metrics);
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan of one 64-bit value per thread (256 threads)
__device__ __forceinline__ long long block_exclusive_scan(long long x, long long* total) {
    __shared__ long long warp_sum[LANESCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    long long base = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < LANESCAN_THREADS / 32; ++w) {
        const long long ws = warp_sum[w];
        if (w < warp) base += ws;
        tot += ws;
    }
    __syncthreads();
    *total = tot;
    return base + incl - x;
}

// k_lanescan.  Tickets [0, n_lane_tiles): next-snapshot lane offsets.
// newsize(l) = size(l) - leave(l) + enter(l); two exclusive prefix sums (new
// sizes, leavers) over lanes in one decoupled look-back pass; tile words pack
// (flag:2 | leavers:31 | sizes:31).  Ticket n_lane_tiles: exclusive prefix of
// the leavers per slot tile.  Remaining tickets: signal states of the next
// step for chunks of junctions.
template <typename Real>
__global__ void __launch_bounds__(LANESCAN_THREADS) k_lanescan(Ctx<Real> c) {
    if (c.cnt->err & ERR_POISON) return;
    __shared__ int s_tile;
    __shared__ unsigned long long s_prefix;
    const int n_tickets = c.n_lane_tiles + 1 + c.n_junc_chunks;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&c.cnt->ticket_lane, 1);
        __syncthreads();
        const int tile = s_tile;
        __syncthreads();
        if (tile >= n_tickets) return;
        if (tile < c.n_lane_tiles) {
            const int base = tile * LANESCAN_TILE + threadIdx.x * LANESCAN_ITEMS;
            int ns[LANESCAN_ITEMS], lv[LANESCAN_ITEMS];
            long long tn = 0, tl = 0;
            if (base + LANESCAN_ITEMS <= c.n_lanes) {
                // 16-byte loads (base is a multiple of 4)
                int o[LANESCAN_ITEMS + 1];
#pragma unroll
                for (int k = 0; k < LANESCAN_ITEMS; k += 4) {
                    const int4 ov = *reinterpret_cast<const int4*>(c.cur.off + base + k);
                    const int4 lvv = *reinterpret_cast<const int4*>(c.leave + base + k);
                    const int4 env = *reinterpret_cast<const int4*>(c.enter + base + k);
                    o[k] = ov.x; o[k + 1] = ov.y; o[k + 2] = ov.z; o[k + 3] = ov.w;
                    lv[k] = lvv.x; lv[k + 1] = lvv.y; lv[k + 2] = lvv.z; lv[k + 3] = lvv.w;
                    ns[k] = env.x; ns[k + 1] = env.y; ns[k + 2] = env.z; ns[k + 3] = env.w;
                    *reinterpret_cast<int4*>(c.leave + base + k) = make_int4(0, 0, 0, 0);
                    *reinterpret_cast<int4*>(c.enter + base + k) = make_int4(0, 0, 0, 0);
                }
                o[LANESCAN_ITEMS] = c.cur.off[base + LANESCAN_ITEMS];
#pragma unroll
                for (int k = 0; k < LANESCAN_ITEMS; ++k) ns[k] += o[k + 1] - o[k] - lv[k];
            } else {
#pragma unroll
                for (int k = 0; k < LANESCAN_ITEMS; ++k) {
                    const int l = base + k;
                    if (l < c.n_lanes) {
                        const int sz = c.cur.off[l + 1] - c.cur.off[l];
                        lv[k] = c.leave[l];
                        ns[k] = sz - lv[k] + c.enter[l];
                        c.leave[l] = 0;
                        c.enter[l] = 0;
                    } else {
                        ns[k] = 0; lv[k] = 0;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < LANESCAN_ITEMS; ++k) { tn += ns[k]; tl += lv[k]; }
            const long long packed = (tl << 31) | tn;
            long long total;
            const long long excl_in = block_exclusive_scan(packed, &total);
            if (threadIdx.x < 32) {
                bool timeout = false;
                unsigned long long prefix = 0;
                if (tile == 0) {
                    if (threadIdx.x == 0) store_release(&c.lane_tiles[0], (2ull << 62) | (unsigned long long)total);
                } else {
                    if (threadIdx.x == 0) store_release(&c.lane_tiles[tile], (1ull << 62) | (unsigned long long)total);
                    prefix = warp_lookback(c.lane_tiles, tile, &timeout);
                    if (threadIdx.x == 0) {
                        store_release(&c.lane_tiles[tile], (2ull << 62) | (prefix + (unsigned long long)total));
                        if (timeout) atomicOr(&c.cnt->err, ERR_TIMEOUT);
                    }
                }
                if (threadIdx.x == 0) s_prefix = prefix;
            }
            __syncthreads();
            long long excl = (long long)s_prefix + excl_in;
            long long en = excl & ((1ll << 31) - 1), el = excl >> 31;
#pragma unroll
            for (int k = 0; k < LANESCAN_ITEMS; ++k) {
                const int l = base + k;
                if (l < c.n_lanes) {
                    c.nxt.off[l] = (int)en;
                    c.lbefore[l] = (int)el;
                }
                en += ns[k]; el += lv[k];
            }
            if (tile == c.n_lane_tiles - 1 && threadIdx.x == LANESCAN_THREADS - 1) {
                c.nxt.off[c.n_lanes] = (int)en;
                c.cnt->n_next = (int)en;
            }
        } else if (tile == c.n_lane_tiles) {
            // leavers before each slot tile of the current snapshot: every
            // thread sums a contiguous run of tiles (loads issued together),
            // one block scan, then the runs are written out; the counters are
            // zeroed for the next step
            // (16-byte loads; the arrays are padded to a multiple of 4 * 256
            // entries and hold zeros beyond the tiles in use)
            const int nt = (c.cnt->n_cur + TILE - 1) / TILE;
            const int per4 = (nt + 4 * LANESCAN_THREADS - 1) / (4 * LANESCAN_THREADS);
            const int k0 = threadIdx.x * per4 * 4;
            long long run = 0;
#pragma unroll 4
            for (int q = 0; q < per4; ++q) {
                const int4 x = *reinterpret_cast<const int4*>(c.tile_leave + k0 + 4 * q);
                run += x.x + x.y + x.z + x.w;
            }
            long long tot;
            long long acc = block_exclusive_scan(run, &tot);
            for (int q = 0; q < per4; ++q) {
                const int4 x = *reinterpret_cast<const int4*>(c.tile_leave + k0 + 4 * q);
                int4 p;
                p.x = (int)acc; acc += x.x;
                p.y = (int)acc; acc += x.y;
                p.z = (int)acc; acc += x.z;
                p.w = (int)acc; acc += x.w;
                *reinterpret_cast<int4*>(c.tile_prefix + k0 + 4 * q) = p;
                *reinterpret_cast<int4*>(c.tile_leave + k0 + 4 * q) = make_int4(0, 0, 0, 0);
            }
        } else {
            // signal states of the next step
            const int j0 = (tile - c.n_lane_tiles - 1) * JUNC_CHUNK;
            const int j = j0 + threadIdx.x;
            if (j < c.n_junctions) c.junc_state[j] = junction_state_at(c, j, 1);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_place: writes the next snapshot.  Stayer tiles (one per block iteration):
// a vehicle that kept its lane goes to off'[lane] + (stayers ahead of it in
// the lane) + (entrants ahead of it); stayers ahead = its slot rank in the
// lane minus the leavers before it in the lane.  Then the entrants: rank =
// stayers ahead + entrants ahead.  The last block to finish closes the step.
template <typename Real>
__device__ __forceinline__ int entrants_ahead(const Ctx<Real>& c, int lane, Real s, int id, int tag) {
    int cnt = 0, guard = 0;
    for (int q = list_head(c.head, lane, tag); q >= 0; q = c.enext[q]) {
        const RecA<Real> Q = c.ea[q];
        if (ahead(Q.s, Q.id, s, id)) ++cnt;
        if (++guard > c.n_veh) { atomicOr(&c.cnt->err, ERR_RANGE); break; }
    }
    return cnt;
}

template <typename Real>
__global__ void __launch_bounds__(TILE) k_place(Ctx<Real> c) {
    if (c.cnt->err & ERR_POISON) return;
    __shared__ int s_warp[TILE / 32];
    const int n = c.cnt->n_cur;
    const int n_ent = c.cnt->n_ent;
    const int tag = c.cnt->tag;
    const int n_tiles = (n + TILE - 1) / TILE;
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int i = tile * TILE + threadIdx.x;
        const bool valid = i < n;
        const int8_t code = valid ? c.code[i] : C_STAY;
        RecA<Real> A;
        RecB B;
        SV<Real> w;
        if (valid) {  // issued before the tile's leaver scan
            A = c.cur.a[i];
            B = c.cur.b[i];
            w = c.stay[i];
        }
        const int leaver = (valid && code != C_STAY) ? 1 : 0;
        const unsigned ball = __ballot_sync(0xffffffffu, leaver);
        const int wpre = __popc(ball & ((1u << lane_id) - 1));
        if (lane_id == 0) s_warp[warp] = __popc(ball);
        __syncthreads();
        int wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += s_warp[w];
        __syncthreads();
        if (valid && code == C_STAY) {
            const int lane = A.lane;
            const int leavers_before = c.tile_prefix[tile] + wbase + wpre;
            const int stay_rank = (i - c.cur.off[lane]) - (leavers_before - c.lbefore[lane]);
            const int pos = c.nxt.off[lane] + stay_rank + entrants_ahead(c, lane, w.s, A.id, tag);
            if (pos < c.nxt.off[lane] || pos >= c.nxt.off[lane + 1]) {
                atomicOr(&c.cnt->err, ERR_RANGE);
            } else {
                RecA<Real> O;
                O.s = w.s; O.v = w.v; O.id = A.id; O.lane = lane;
                c.nxt.a[pos] = O;
                c.nxt.b[pos] = B;
            }
        }
    }
    // entrants: one warp per entrant; the warp counts the stayers of the
    // lane's old segment that are ahead of it, 32 slots per round
    const int gwarp = blockIdx.x * (TILE / 32) + warp, nwarps = gridDim.x * (TILE / 32);
    for (int q = gwarp; q < n_ent; q += nwarps) {
        const RecA<Real> Q = c.ea[q];
        const int lane = Q.lane;
        const int b = c.cur.off[lane], e = c.cur.off[lane + 1];
        int rank = 0;
        for (int k = b + lane_id; k - lane_id < e; k += 32) {
            const bool p = k < e && c.code[k] == C_STAY && ahead(c.stay[k].s, c.cur.a[k].id, Q.s, Q.id);
            rank += __popc(__ballot_sync(0xffffffffu, p));
        }
        if (lane_id == 0) {
            rank += entrants_ahead(c, lane, Q.s, Q.id, tag);
            const int pos = c.nxt.off[lane] + rank;
            if (pos < c.nxt.off[lane] || pos >= c.nxt.off[lane + 1]) {
                atomicOr(&c.cnt->err, ERR_RANGE);
            } else {
                c.nxt.a[pos] = Q;
                c.nxt.b[pos] = c.eb[q];
            }
        }
    }
    // clear the lane look-back words for the next step (k_lanescan is done)
    for (int k = blockIdx.x * TILE + threadIdx.x; k < c.n_lane_tiles; k += gridDim.x * TILE)
        c.lane_tiles[k] = 0ull;
    // the last block to finish closes the step: publish the next snapshot
    // size, reset the step counters, advance the list tag and every
    // scenario's clock
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(&c.cnt->done_place, 1);
        if (done == (int)gridDim.x - 1) {
            __threadfence();
            c.cnt->n_cur = c.cnt->n_next;
            c.cnt->n_ent = 0;
            c.cnt->ticket_lane = 0;
            c.cnt->done_place = 0;
            int tg = c.cnt->tag + 1;
            c.cnt->tag = tg > 0x3fffffff ? 1 : tg;
            for (int s = 0; s < c.n_scen; ++s) c.scen_step[s] += 1;
            __threadfence();
        }
    }
}

// signal states for the current step of every junction (after creation or
// a state reset)
template <typename Real>
__global__ void k_junction_init(Ctx<Real> c) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < c.n_junctions; j += gridDim.x * blockDim.x)
        c.junc_state[j] = junction_state_at(c, j, 0);
}

// setter: policy (and manual phase) of n junctions, effective from the
// current step (the state of the step is recomputed)
template <typename Real>
__global__ void k_set_signal(Ctx<Real> c, int n, const int32_t* ids, const int32_t* phases, int policy) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int j = ids[k];
    c.junc_policy[j] = policy;
    if (policy == POL_MANUAL) c.junc_manual[j] = phases[k];
    c.junc_state[j] = junction_state_at(c, j, 0);
}

// Failure-detection self-test: the look-back of tile 1 waits on tile word 0,
// which nothing publishes, so the bounded wait must give up and report.
__global__ void k_selftest_wait(unsigned long long* words, int* err) {
    bool timeout = false;
    warp_lookback(words, 1, &timeout);
    if (threadIdx.x == 0 && timeout) atomicOr(err, ERR_TIMEOUT);
}

}  // namespace moss
