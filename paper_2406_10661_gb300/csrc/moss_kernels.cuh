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
// A k_decide block's lane-change candidates: their indices in the candidate
// list, resolved by the block once its run is done; past cand_cap of them (a
// schedule value, at most CAND_LOCAL) the rest go to the late list that
// k_lanescan's first tickets resolve.
constexpr int CAND_LOCAL = 256;
struct CandLocal {
    int n;
    int idx[CAND_LOCAL];
};

template <typename Real>
__device__ __forceinline__ void note_candidate(const Ctx<Real>& c, CandLocal& cl, int k) {
    const int j = atomicAdd(&cl.n, 1);
    if (j < c.cand_cap) cl.idx[j] = k;
    else c.cand_late[atomicAdd(&c.cnt->n_late, 1)] = k;
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
    const LaneInfo ls = c.lane[l];
    if (ls.flags & LF_RESTRICTED) return;  // no departure onto a restricted lane (R25)
    const int sc = ls.scen;
    if (c.scen_ctl[sc]) return;  // a frozen or retiring slot
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
    const int q = warp_claim(&c.cnt->n_ent);
    const int2 rs = c.route_span[vid];
    const int r0 = rs.x, r1 = rs.y - 1;
    int nl = -1;
    if (r0 < r1) nl = jl_toward(c, c.lane[l], c.routes[r0 + 1]);  // -1: no access from this lane (R27)
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
            if (++iter > 4 || nl < 0) { atomicOr(c.err, ERR_TRANSFER); sn = Ll; break; }
            sn = ex;
            fl |= F_TRANSFER;
            nlane = nl;
            ni = c.lane[nlane];
            if (road) {
                nl = ni.hi;  // entered a junction lane: next is its target road lane
            } else {
                rptr += 1;  // entered the next road
                // -1 on the last road, or without access from this lane (R27)
                nl = (rptr < rlast) ? jl_toward(c, ni, c.routes[rptr + 1]) : -1;
            }
            ex = sn - Real(ni.L);
        }
    }
    if (arrived) fl |= F_ARRIVED;
    acc.upd += 1;
    acc.spd += speed_fixed(vn);
    if (fl & F_FLAGGED) acc.flg += 1;
    if (fl & F_CHANGED) acc.lc += 1;
    if (own_overlap) acc.ovl += 1;
    if (fl) c.vflags[E.id] = int((t & 0xFFFFFF) << 8) | fl;
    if (arrived) {
        c.code[i] = C_ARRIVE;
        c.vstatus[E.id] = 2;
        acc.arr += 1;
        acc.tt += (t + 1) - (long long)c.dep[E.id];
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
    const int q = warp_claim(&c.cnt->n_ent);
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
// A lane-change candidate leaves its decision for k_resolve: a record in the
// candidate list, linked into the list of its target gap.
template <typename Real>
__device__ __forceinline__ void list_candidate(const Ctx<Real>& c, int i, const RecA<Real>& E, const RecB& EB,
                                               int sc, const Decision<Real>& D, int tag, CandLocal& cl) {
    int gp;
    if (D.TF >= 0) gp = D.TF;
    else if (D.TL >= 0) gp = D.TL + 1;
    else gp = c.cur.off[D.tl];
    const LaneInfo ti = c.lane[D.tl];
    RecA<Real> TLr;
    TLr.s = Real(0); TLr.v = Real(0);
    if (D.TL >= 0) TLr = c.cur.a[D.TL];
    const LaneAcc<Real> T = accel_on_lane(c, ti, E.s, E.v, Real(EB.v0f) * Real(ti.vmax), D.TL >= 0, TLr.s, TLr.v,
                                          D.nlt, EB.rptr, EB.rlast);
    Cand<Real> C;
    C.E = E; C.EB = EB;
    C.slot = i; C.gap = gp + D.tl;
    C.bits = (D.dir > 0 ? CB_RIGHT : 0) | (D.flag ? CB_FLAG : 0) | (D.own.has_leader ? CB_LEADER : 0) |
             (D.own.stop ? CB_STOP : 0) | (D.own.overlap ? CB_OVERLAP : 0) | (T.has_leader ? CB_TLEADER : 0) |
             (T.stop ? CB_TSTOP : 0) | (T.overlap ? CB_TOVERLAP : 0);
    C.nl = D.own.nl; C.tnl = T.nl; C.scen = sc; C.pad = 0;
    C.u = D.u; C.scale = D.scale;
    C.a = D.own.a; C.lgap = D.own.gap; C.sgap = D.own.stop_gap;
    C.ta = T.a; C.tlgap = T.gap; C.tsgap = T.stop_gap;
    const int k = warp_claim(&c.cnt->n_cand);
    const unsigned long long prev =
        atomicExch(&c.gap_head[C.gap], ((unsigned long long)(unsigned)tag << 32) | (unsigned)k);
    C.next = (int)(prev >> 32) == tag ? (int)(unsigned)(prev & 0xffffffffull) : -1;
    c.cands[k] = C;
    note_candidate(c, cl, k);
}

// ---------------------------------------------------------------------------
// Resolution of lane-change candidate k.  Conflict rule R9: a candidate
// conflicts with the candidates that enter the same lane from the other side
// into the same gap
// (the other members of its gap list with the opposite direction); the
// larger utility wins, ties to the smaller id.  Both sides compare the same
// stored utilities, so the outcome is consistent.  Then the update on the
// target lane (granted) or with the stored own-lane kinematics (lost).
template <typename Real>
__device__ __forceinline__ void resolve_one(const Ctx<Real>& c, MetricAcc& acc, int k, int nc, int tag) {
    {
        const Cand<Real> C = c.cands[k];
        const int i = C.slot;
        const RecA<Real> E = C.E;
        const RecB EB = C.EB;
        const int lane = E.lane;
        const int dir = (C.bits & CB_RIGHT) ? 1 : -1;
        const int sc = C.scen;
        if (sc != acc.scen) {
            macc_flush_thread(acc, c.metrics);
            macc_reset(acc, sc);
        }
        const long long t = c.scen_step[sc];
        int fl = F_CANDIDATE | ((C.bits & CB_FLAG) ? F_FLAGGED : 0);
        bool granted = true;
        const unsigned long long h = c.gap_head[C.gap];
        int q = (int)(h >> 32) == tag ? (int)(unsigned)(h & 0xffffffffull) : -1;
        for (int guard = 0; q >= 0; q = c.cands[q].next) {
            if (++guard > nc) { atomicOr(c.err, ERR_RANGE); break; }
            if (q == k) continue;
            const int rbits = c.cands[q].bits;
            if (((rbits & CB_RIGHT) ? 1 : -1) == dir) continue;  // same side: no conflict
            const Real ru = c.cands[q].u, rs = c.cands[q].scale;
            const Real sc2 = C.scale > rs ? C.scale : rs;
            if (rabs(C.u - ru) < c.band * sc2) fl |= F_FLAGGED;
            if (!(C.u > ru || (C.u == ru && E.id < c.cands[q].E.id))) granted = false;
        }
        LaneAcc<Real> la;
        int nlane = lane;
        if (granted) {
            fl |= F_CHANGED;
            nlane = lane + dir;
            la.a = C.ta; la.gap = C.tlgap; la.stop_gap = C.tsgap; la.nl = C.tnl;
            la.has_leader = (C.bits & CB_TLEADER) != 0;
            la.stop = (C.bits & CB_TSTOP) != 0;
            la.overlap = (C.bits & CB_TOVERLAP) != 0;
        } else {
            fl |= F_CONFLICT_LOST;
            la.a = C.a; la.gap = C.lgap; la.stop_gap = C.sgap; la.nl = C.nl;
            la.has_leader = (C.bits & CB_LEADER) != 0;
            la.stop = (C.bits & CB_STOP) != 0;
            la.overlap = (C.bits & CB_OVERLAP) != 0;
        }
        integrate_emit(c, acc, i, E, EB, la, nlane, fl, (C.bits & CB_OVERLAP) != 0, t, sc, tag);
    }
}

// ---------------------------------------------------------------------------
// The vehicles whose attempt draw passed are queued in shared memory, one
// queue of 64 entries per warp, and MOBIL runs over a warp's queue 32 at a
// time: a warp otherwise carries the whole MOBIL evaluation of any one of
// its lanes while the others idle.
template <typename Real>
struct MobilQueue {
    Real a[2 * TILE], gap[2 * TILE], sgap[2 * TILE];  // own-lane kinematics (LaneAcc)
    int i[2 * TILE], lane[2 * TILE], bits[2 * TILE], nl[2 * TILE];
    float u_lc[2 * TILE], u_dir[2 * TILE];
    int n[TILE / 32];
};

// MOBIL and the update of queued vehicle k (the snapshot and lane records
// are read again; the own-lane part comes from the queue)
template <typename Real, bool Groups>
__device__ __forceinline__ void mobil_finish(const Ctx<Real>& c, const MobilQueue<Real>& q, int k, int n,
                                             MetricAcc& acc, int tag, CandLocal& cl) {
    const int i = q.i[k], lane = q.lane[k];
    const RecA<Real> E = c.cur.a[i];
    const RecB EB = c.cur.b[i];
    const LaneInfo li = c.lane[lane];
    RecA<Real> OLr = no_rec<Real>(), OFr = no_rec<Real>();
    float of_v0f = 0.0f;
    if (i > 0) OLr = c.cur.a[i - 1];
    if (i + 1 < n) {
        OFr = c.cur.a[i + 1];
        of_v0f = c.cur.b[i + 1].v0f;
    }
    LaneAcc<Real> own;
    own.a = q.a[k]; own.gap = q.gap[k]; own.stop_gap = q.sgap[k];
    const int bits = q.bits[k];
    own.has_leader = bits & 1; own.stop = (bits >> 1) & 1; own.overlap = (bits >> 2) & 1;
    own.nl = q.nl[k];
    const int sc = li.scen;
    if (sc != acc.scen) {
        macc_flush_thread(acc, c.metrics);
        macc_reset(acc, sc);
    }
    const Decision<Real> D = decide_mobil<Real, Groups>(c, E, EB, li, OLr, OFr, of_v0f, own, q.u_lc[k], q.u_dir[k]);
    if (D.cand) {
        list_candidate(c, i, E, EB, sc, D, tag, cl);
        return;
    }
    const long long t = c.scen_step[sc];
    integrate_emit(c, acc, i, E, EB, own, lane, D.flag ? F_FLAGGED : 0, own.overlap != 0, t, sc, tag);
}

// ---------------------------------------------------------------------------
// k_decide: blocks [0, n_work) take 256-slot tiles of the current snapshot
// (one vehicle per thread); blocks [n_work, gridDim) run the insertion.
// Per vehicle: the own-lane acceleration and the attempt draw, MOBIL if the
// draw passed (from the warp's queue, above), then the update; lane-change
// candidates are finished by k_resolve.
// Groups: the network has lane groups (some road has a turn that not all of
// its lanes serve), so the mandatory changes of R27 can occur; without them
// that path is not compiled in.
// MOSS_DECIDE_MIN_BLOCKS: resident blocks per SM the register budget targets.
#ifndef MOSS_DECIDE_MIN_BLOCKS
#define MOSS_DECIDE_MIN_BLOCKS 5
#endif
// The run of slots [*sb, *se) of work block vb of n_work.  A vehicle on a
// road lane costs about twice one on a junction lane (MOBIL, longer
// neighbour searches), so the runs split the snapshot by weight: run_w (a
// schedule choice, 2 by default) per road-lane slot, 1 per junction-lane
// slot, from the current lane offsets at the lane ranges of each scenario
// (road lanes first, then junction lanes), when blocks take four tiles or
// more each; then each end moves back to the start of its road.  The runs
// are contiguous and cover every slot.
__device__ __forceinline__ long long run_weight(int a, int b, int e, int wq) {
    return (long long)wq * (b - a) + 256ll * (e - b);
}
// road-lane slot weight x256 of this step's runs: the schedule's fixed value,
// else the fit of the previous step's block times (1 before any)
template <typename Real>
__device__ __forceinline__ int run_wq(const Ctx<Real>& c) {
    if (c.run_w > 0) return 256 * c.run_w;
    const int f = c.cnt->run_wq;
    return f > 0 ? f : 256;
}

// First slot of the road whose lane holds `slot` (a junction-lane slot
// stays where it is): the block runs begin and end there, so the vehicles of
// a road, and with them every rival of a lane-change candidate, lie in one run.
template <typename Real>
__device__ __forceinline__ int road_start(const Ctx<Real>& c, int slot, int n) {
    if (slot <= 0) return 0;
    if (slot >= n) return n;
    const int lane = c.cur.a[slot].lane;
    if ((unsigned)lane >= (unsigned)c.n_lanes) return slot;  // reported by the decision
    const int lo = c.lane[lane].lo;
    return lo >= 0 ? c.cur.off[lo] : slot;
}

template <typename Real>
__device__ __forceinline__ void decide_run(const Ctx<Real>& c, int n, int n_work, int vb, int* sb, int* se) {
    __shared__ int s_run[2];
    const int n_tiles = (n + TILE - 1) / TILE;
    if (n_tiles < 4 * n_work) {
        // a few tiles per block: equal slot counts (weights would leave
        // blocks idle at this granularity)
        if (threadIdx.x == 0) {
            s_run[0] = road_start(c, (int)((long long)vb * n / n_work), n);
            s_run[1] = road_start(c, (int)((long long)(vb + 1) * n / n_work), n);
        }
    } else if (threadIdx.x < 32) {
        const int wl = threadIdx.x;
        const int wq = run_wq(c);
        long long tot = 0;
        for (int k0 = 0; k0 < c.n_scen; k0 += 32) {
            long long w = 0;
            if (k0 + wl < c.n_scen) {
                const int4 L = c.scen_lanes[k0 + wl];
                w = run_weight(c.cur.off[L.x], c.cur.off[L.y], c.cur.off[L.z], wq);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            tot += w;
        }
        // weights T0, T1 -> slots (scan of the scenarios' weights)
        const long long T[2] = {tot * vb / n_work, tot * (vb + 1) / n_work};
        int slot[2] = {-1, -1};
        long long carry = 0;
        for (int k0 = 0; k0 < c.n_scen && (slot[0] < 0 || slot[1] < 0); k0 += 32) {
            const int k = k0 + wl;
            int a = 0, b = 0, e = 0;
            long long w = 0;
            if (k < c.n_scen) {
                const int4 L = c.scen_lanes[k];
                a = c.cur.off[L.x]; b = c.cur.off[L.y]; e = c.cur.off[L.z];
                w = run_weight(a, b, e, wq);
            }
            long long P = w;  // inclusive prefix over the chunk
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, P, o);
                if (wl >= o) P += y;
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                // the first scenario whose weight reaches past T (m and
                // slot[q] are the same on every lane: the branch is uniform)
                const unsigned m = __ballot_sync(0xffffffffu, k < c.n_scen && carry + P > T[q]);
                if (slot[q] < 0 && m) {
                    const int src = __ffs(m) - 1;
                    const long long local = T[q] - (carry + __shfl_sync(0xffffffffu, P - w, src));
                    const int sa = __shfl_sync(0xffffffffu, a, src), sb = __shfl_sync(0xffffffffu, b, src);
                    const long long wr = (long long)wq * (sb - sa);
                    slot[q] = local < wr ? sa + (int)(local / wq) : sb + (int)((local - wr) / 256);
                }
            }
            carry += __shfl_sync(0xffffffffu, P, 31);
        }
        if (wl == 0) {
            const int s0 = slot[0] < 0 ? n : slot[0], s1 = slot[1] < 0 ? n : slot[1];
            s_run[0] = road_start(c, s0, n);
            s_run[1] = vb == n_work - 1 ? n : road_start(c, s1, n);
        }
    }
    __syncthreads();
    *sb = s_run[0];
    *se = s_run[1];
}

// The work of block vb of nvb (k_decide's grid, or a virtual block of the
// single-launch step): vb < n_work takes a run of slot tiles, the others run
// the insertion.
template <typename Real, bool Groups>
__device__ __forceinline__ void decide_block(const Ctx<Real>& c, int n_work, int vb, int nvb) {
    const int tag = c.cnt->tag;
    if (vb >= n_work) {
        const int stride = (nvb - n_work) * TILE;
        for (int k = (vb - n_work) * TILE + threadIdx.x; k < c.n_start; k += stride)
            insert_departure(c, c.start_lanes[k], tag);
        return;
    }
    const int n = c.cnt->n_cur;
    // each block takes a contiguous run of slots: a thread's scenario (and so
    // its metric partials) changes rarely, neighbouring lanes stay close, and
    // the run holds whole roads, so the block resolves its own lane-change
    // candidates once its run is done (rule R9: rivals share the road)
    __shared__ CandLocal cl;
    __shared__ MobilQueue<Real> q;
    __shared__ int s_road;  // road-lane vehicles of the run (for the run-weight fit)
    unsigned long long t_start = 0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
    if (threadIdx.x == 0) { cl.n = 0; s_road = 0; }
    if (vb == 0 && threadIdx.x == 0) c.cnt->n_runs = n_work;
    int n_road = 0;
    int s_beg, s_end;
    decide_run(c, n, n_work, vb, &s_beg, &s_end);
    const int t_beg = s_beg / TILE, t_end = s_beg < s_end ? (s_end + TILE - 1) / TILE : t_beg;
    MetricAcc acc;
    macc_reset(acc, -1);
    const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31, qb = warp * 64;
    if (wl == 0) q.n[warp] = 0;
    __syncwarp();
    for (int tile = t_beg;; ++tile) {
        const bool last = tile >= t_end;
        const int i = tile * TILE + threadIdx.x;
        if (!last && i >= s_beg && i < s_end) {
            const RecA<Real> E = c.cur.a[i];
            const RecB EB = c.cur.b[i];
            const RecA<Real> OLr = i > 0 ? c.cur.a[i - 1] : no_rec<Real>();
            const int lane = E.lane;
            if ((unsigned)lane >= (unsigned)c.n_lanes) {
                atomicOr(c.err, ERR_RANGE);
            } else {
                const LaneInfo li = c.lane[lane];
                n_road += li.lo >= 0;
                const int sc = li.scen;
                if (sc != acc.scen) {
                    macc_flush_thread(acc, c.metrics);
                    macc_reset(acc, sc);
                }
                const int ctl = c.scen_ctl[sc];
                if (ctl) {
                    // a slot that does not advance: a frozen one keeps its
                    // vehicles as they are, a retiring one removes them
                    if (ctl & SC_RETIRE) {
                        c.code[i] = C_ARRIVE;
                        c.vstatus[E.id] = 2;
                        atomicAdd(&c.leave[lane], 1);
                    } else {
                        c.code[i] = C_STAY;
                        SV<Real> w;
                        w.s = E.s; w.v = E.v;
                        c.stay[i] = w;
                    }
                } else {
                    const long long t = c.scen_step[sc];
                    const OwnPart<Real> P =
                        decide_own<Real, Groups>(c, E, EB, li, OLr, t, c.key0[sc], c.key1[sc], c.veh_base[sc]);
                    int fl = 0;
                    bool cand = false;
                    if (P.att) {
                        acc.mob += 1;
                        const int k = qb + warp_claim(&q.n[warp]);
                        q.i[k] = i; q.lane[k] = lane;
                        q.a[k] = P.own.a; q.gap[k] = P.own.gap; q.sgap[k] = P.own.stop_gap;
                        q.bits[k] = (P.own.has_leader ? 1 : 0) | (P.own.stop ? 2 : 0) | (P.own.overlap ? 4 : 0);
                        q.nl[k] = P.own.nl;
                        q.u_lc[k] = P.u_lc; q.u_dir[k] = P.u_dir;
                        cand = true;  // finished from the queue
                    } else if (Groups && P.mand) {
                        const Decision<Real> D = decide_mandatory(c, i, E, EB, li, P.own);
                        if (D.cand) {
                            list_candidate(c, i, E, EB, sc, D, tag, cl);
                            cand = true;
                        }
                        fl = D.flag ? F_FLAGGED : 0;
                    }
                    if (!cand) integrate_emit(c, acc, i, E, EB, P.own, lane, fl, P.own.overlap != 0, t, sc, tag);
                }
            }
        }
        // MOBIL over the last 32 entries of the warp's queue once it holds
        // 32, and over what is left after the last tile
        __syncwarp();
        const int nq = q.n[warp];
        const int take = last ? nq : (nq >= 32 ? 32 : 0);
        if (take > 0) {
            if (wl < take) mobil_finish<Real, Groups>(c, q, qb + nq - take + wl, n, acc, tag, cl);
            __syncwarp();
            if (wl == 0) q.n[warp] = nq - take;
            __syncwarp();
        }
        if (last) break;
    }
    // the run's lane-change candidates (their rivals are all in this run)
    __syncthreads();
    const int ncl = min(cl.n, c.cand_cap);
    for (int j = threadIdx.x; j < ncl; j += TILE) resolve_one(c, acc, cl.idx[j], c.n_veh, tag);
    if (n_road) atomicAdd(&s_road, n_road);
    macc_flush_block<TILE>(acc, c.metrics);  // (its barriers also complete s_road)
    // the run's statistics for the next step's weight fit (run_fit)
    if (threadIdx.x == 0 && vb < RUNSTAT_MAX) {
        unsigned long long t_end = 0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
        const long long dt = (long long)(t_end - t_start);
        const int ns = s_end - s_beg;
        c.runstat[vb] = make_int4((int)min(dt, (long long)INT_MAX), s_road, ns - s_road, 1);
    }
}

template <typename Real, bool Groups>
__global__ void __launch_bounds__(TILE, MOSS_DECIDE_MIN_BLOCKS) k_decide(Ctx<Real> c, int n_work) {
    if (*c.err & ERR_POISON) return;
    decide_block<Real, Groups>(c, n_work, blockIdx.x, gridDim.x);
}

template <typename Real>
__global__ void __launch_bounds__(TILE) k_resolve(Ctx<Real> c) {
    if (*c.err & ERR_POISON) return;
    const int nc = c.cnt->n_late;
    const int tag = c.cnt->tag;
    MetricAcc acc;
    macc_reset(acc, -1);
    for (int k = blockIdx.x * TILE + threadIdx.x; k < nc; k += gridDim.x * TILE)
        resolve_one(c, acc, c.cand_late[k], c.n_veh, tag);
    // the phase pressures of the max-pressure junctions (read by k_lanescan)
    if (*c.n_mp > 0)
        for (int k = blockIdx.x * TILE + threadIdx.x; k < c.n_jj; k += gridDim.x * TILE) mp_accumulate(c, k);
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

// One lane tile of k_lanescan (LS_ROUNDS x 1024 lanes).  newsize(l) =
// size(l) - leave(l) + enter(l); its exclusive prefix sum over lanes (the
// next lane offsets) in one decoupled look-back pass; tile words pack
// (flag:2 | sum:62).  Warp w takes LS_ROUNDS x 128 consecutive lanes of the
// tile in LS_ROUNDS rounds of 128 (4 consecutive lanes per thread), so each
// 16-byte load and store of a warp covers one contiguous 512-byte run.  The
// tile size is a schedule choice (moss_autotune): 4 rounds (4096 lanes) or 2.
constexpr int LS_WARPS = LANESCAN_THREADS / 32;
static_assert(LANESCAN_TILE == LS_WARPS * 128 * 4, "the default lane tile has 4 rounds");
static_assert(JUNC_CHUNK == LANESCAN_THREADS, "one junction per thread");

template <typename Real, int LS_ROUNDS>
__device__ __forceinline__ void lanescan_tile(const Ctx<Real>& c, int tile) {
    constexpr int LS_TILE = LS_WARPS * 128 * LS_ROUNDS;
    __shared__ long long s_wsum[LS_WARPS];
    __shared__ unsigned long long s_prefix;
    const int ln = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nl = c.n_lanes;
    const int wbase = tile * LS_TILE + w * (LS_TILE / LS_WARPS);
    int ns[LS_ROUNDS][4];
    long long wpre[LS_ROUNDS];
    long long run = 0;
    // every load of the tile is issued before any result is used (and before
    // the zeroing stores), so the tile costs one memory round trip
    int o[LS_ROUNDS][4], lvv[LS_ROUNDS][4], env[LS_ROUNDS][4], o4[LS_ROUNDS];
#pragma unroll
    for (int r = 0; r < LS_ROUNDS; ++r) {
        const int l0 = wbase + r * 128 + 4 * ln;
        if (l0 + 4 <= nl) {
            const int4 ov = *reinterpret_cast<const int4*>(c.cur.off + l0);
            const int4 lx = *reinterpret_cast<const int4*>(c.leave + l0);
            const int4 ex = *reinterpret_cast<const int4*>(c.enter + l0);
            o[r][0] = ov.x; o[r][1] = ov.y; o[r][2] = ov.z; o[r][3] = ov.w;
            lvv[r][0] = lx.x; lvv[r][1] = lx.y; lvv[r][2] = lx.z; lvv[r][3] = lx.w;
            env[r][0] = ex.x; env[r][1] = ex.y; env[r][2] = ex.z; env[r][3] = ex.w;
            o4[r] = ln == 31 ? c.cur.off[l0 + 4] : 0;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int l = l0 + j;
                const bool in = l < nl;
                o[r][j] = in || l == nl ? c.cur.off[l] : 0;
                lvv[r][j] = in ? c.leave[l] : 0;
                env[r][j] = in ? c.enter[l] : 0;
            }
            o4[r] = 0;
        }
    }
#pragma unroll
    for (int r = 0; r < LS_ROUNDS; ++r) {
        const int l0 = wbase + r * 128 + 4 * ln;
        if (l0 + 4 <= nl) {
            *reinterpret_cast<int4*>(c.leave + l0) = make_int4(0, 0, 0, 0);
            *reinterpret_cast<int4*>(c.enter + l0) = make_int4(0, 0, 0, 0);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (l0 + j < nl) { c.leave[l0 + j] = 0; c.enter[l0 + j] = 0; }
        }
    }
#pragma unroll
    for (int r = 0; r < LS_ROUNDS; ++r) {
        const int l0 = wbase + r * 128 + 4 * ln;
        // offset after the thread's 4th lane: the next thread's first
        int onx = __shfl_down_sync(0xffffffffu, o[r][0], 1);
        if (ln == 31) onx = o4[r];
        long long rs = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool valid = l0 + j < nl;
            const int onext = j < 3 ? o[r][j + 1] : onx;
            ns[r][j] = valid ? (onext - o[r][j]) - lvv[r][j] + env[r][j] : 0;
            rs += ns[r][j];
        }
        const long long p = rs;
        long long incl = p;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, incl, d);
            if (ln >= d) incl += y;
        }
        wpre[r] = run + incl - p;
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (ln == 0) s_wsum[w] = run;
    __syncthreads();
    long long wb = 0, total = 0;
#pragma unroll
    for (int k = 0; k < LS_WARPS; ++k) {
        const long long x = s_wsum[k];
        if (k < w) wb += x;
        total += x;
    }
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
                if (timeout) atomicOr(c.err, ERR_TIMEOUT);
            }
        }
        if (threadIdx.x == 0) s_prefix = prefix;
    }
    __syncthreads();
    const long long base = (long long)s_prefix + wb;
#pragma unroll
    for (int r = 0; r < LS_ROUNDS; ++r) {
        const int l0 = wbase + r * 128 + 4 * ln;
        const long long ex = base + wpre[r];
        long long en = ex;
        int on[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            on[j] = (int)en;
            en += ns[r][j];
        }
        if (l0 + 4 <= nl) {
            *reinterpret_cast<int4*>(c.nxt.off + l0) = make_int4(on[0], on[1], on[2], on[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (l0 + j < nl) c.nxt.off[l0 + j] = on[j];
        }
        if (l0 < nl && nl <= l0 + 4) {  // this thread holds the last lane
            c.nxt.off[nl] = (int)en;
            c.cnt_next->n_cur = (int)en;
        }
    }
}

// Fit of the cost of a road-lane and a junction-lane vehicle in k_decide
// from this step's work blocks: least squares of run time ~ c_road x (road
// slots) + c_junction x (junction slots) over the runs; the next step splits
// its runs with the weight c_road / c_junction (clamped to [0.5, 4]; the
// previous weight when the fit is degenerate, e.g. no junction vehicles).
// One block (a ticket of k_lanescan); every work run rewrites its entry each
// step.
template <typename Real>
__device__ void run_fit(const Ctx<Real>& c) {
    // FP32 sums of normalised values (slots in thousands, times in units of
    // 100 us): the five sums stay within a few thousand for any run count
    __shared__ float s_sum[5][TILE / 32];
    float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // RR, RJ, JJ, dR, dJ
    const int nr = min(c.cnt->n_runs, RUNSTAT_MAX);
    for (int k = threadIdx.x; k < nr; k += TILE) {
        const int4 r = c.runstat[k];
        if (!r.w) continue;
        const float d = 1e-5f * (float)r.x, R = 1e-3f * (float)r.y, J = 1e-3f * (float)r.z;
        v[0] += R * R; v[1] += R * J; v[2] += J * J; v[3] += d * R; v[4] += d * J;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        float x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) s_sum[q][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t[5];
        for (int q = 0; q < 5; ++q) {
            t[q] = 0.f;
            for (int w = 0; w < TILE / 32; ++w) t[q] += s_sum[q][w];
        }
        int wq = c.cnt->run_wq;
        const float det = t[0] * t[2] - t[1] * t[1];
        if (det > 1e-4f * t[0] * t[2] && t[2] > 0.f) {
            const float cr = (t[3] * t[2] - t[4] * t[1]) / det, cj = (t[0] * t[4] - t[1] * t[3]) / det;
            if (cr > 0.f && cj > 0.f) {
                const float w = fminf(4.f, fmaxf(0.5f, cr / cj));
                wq = (int)(w * 256.f + 0.5f);
            }
        }
        c.cnt_next->run_wq = wq;
    }
}

// k_lanescan.  Ticket 0: the run-weight fit.  Then (the first tickets below)
// the late candidates and max-pressure sums, the next-snapshot lane offsets
// (lane tiles, above), and the signal states of the next step for chunks of
// junctions.
template <typename Real, int LS_ROUNDS = 4>
__device__ __forceinline__ void lanescan_blocks(const Ctx<Real>& c) {
    __shared__ int s_tile;
#if MOSS_FOLD_RESOLVE
    // first tickets: the lane-change candidates (k_resolve's work) and the
    // max-pressure sums, in chunks of TILE; the later tickets wait until all
    // of those are done (their blocks hold earlier tickets, so they are
    // running: the wait is bounded)
    __shared__ int s_ready;
    const int nc = c.cnt->n_late;  // candidates past the k_decide blocks' own lists
    const int tag = c.cnt->tag;
    const int r_cand = (nc + TILE - 1) / TILE;
    const int n_res = r_cand + (*c.n_mp > 0 ? (c.n_jj + TILE - 1) / TILE : 0);
    if (threadIdx.x == 0) s_ready = n_res == 0;
#else
    const int n_res = 0;
#endif
    const int n_tickets = 1 + n_res + c.n_lane_tiles + c.n_junc_chunks;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&c.cnt->ticket_lane, 1);
        __syncthreads();
        int tile = s_tile;
        __syncthreads();
        if (tile >= n_tickets) return;
        // ticket 0: the run-weight fit of k_decide's runs (needs nothing else)
        if (tile == 0) {
            run_fit(c);
            __syncthreads();
            continue;
        }
        tile -= 1;
#if MOSS_FOLD_RESOLVE
        if (tile < n_res) {
            MetricAcc acc;
            macc_reset(acc, -1);
            if (tile < r_cand) {
                const int k = tile * TILE + threadIdx.x;
                if (k < nc) resolve_one(c, acc, c.cand_late[k], c.n_veh, tag);
            } else {
                const int k = (tile - r_cand) * TILE + threadIdx.x;
                if (k < c.n_jj) mp_accumulate(c, k);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&c.cnt->res_done, 1);
            }
            // the metric sums are read by no later ticket: after the signal
            macc_flush_block<TILE>(acc, c.metrics);
            continue;
        }
        // lane tiles read the enter / leave counts the candidates change;
        // junction tickets read only the max-pressure sums
        if (!s_ready && (tile - n_res < c.n_lane_tiles || *c.n_mp > 0)) {
            if (threadIdx.x == 0) {
                cuda::atomic_ref<int, cuda::thread_scope_device> done(c.cnt->res_done);
                long long spins = 0;
                while (done.load(cuda::memory_order_acquire) < n_res) {
                    if (++spins > SPIN_LIMIT) { atomicOr(c.err, ERR_TIMEOUT); break; }
                    if (spins > 16) __nanosleep(64);
                }
                s_ready = 1;
            }
            __syncthreads();
        }
        tile -= n_res;
#endif
        if (tile < c.n_lane_tiles) {
            lanescan_tile<Real, LS_ROUNDS>(c, tile);
        } else {
            // signal states of the next step
            const int j0 = (tile - c.n_lane_tiles) * JUNC_CHUNK;
            const int j = j0 + threadIdx.x;
            if (j < c.n_junctions && !c.scen_ctl[c.junc[j].scen])
                c.junc_state[j] = c.junc_policy[j] == POL_MAXP ? mp_advance(c, j) : junction_state_at(c, j, 1);
        }
        __syncthreads();
    }
}

template <typename Real, int LS_ROUNDS>
__global__ void __launch_bounds__(LANESCAN_THREADS) k_lanescan(Ctx<Real> c) {
    if (*c.err & ERR_POISON) return;
    lanescan_blocks<Real, LS_ROUNDS>(c);
}

// ---------------------------------------------------------------------------
// k_place: writes the next snapshot.  Stayer tiles (one per block iteration):
// a vehicle that kept its lane goes to off'[lane] + (stayers ahead of it in
// the lane) + (entrants ahead of it), its stayers ahead counted in its tile
// (below).  Then the entrants: rank = stayers ahead + entrants ahead.  Block
// 0 prepares the next step's counters and advances the scenarios' clocks.
template <typename Real>
__device__ __forceinline__ int entrants_ahead(const Ctx<Real>& c, int lane, Real s, int id, int tag,
                                              int* n_in = nullptr) {
    int cnt = 0, guard = 0;
    for (int q = list_head(c.head, lane, tag); q >= 0; q = c.enext[q]) {
        const RecA<Real> Q = c.ea[q];
        if (ahead(Q.s, Q.id, s, id)) ++cnt;
        if (++guard > c.n_veh) { atomicOr(c.err, ERR_RANGE); break; }
    }
    if (n_in) *n_in = guard;
    return cnt;
}

template <typename Real>
__device__ __forceinline__ void place_blocks(const Ctx<Real>& c, int vb, int nvb) {
    __shared__ int s_warp[TILE / 32];
    const int n = c.cnt->n_cur;
    const int n_ent = c.cnt->n_ent;
    const int tag = c.cnt->tag;
    const int n_tiles = (n + TILE - 1) / TILE;
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // closing the step: the next step's counters (k_lanescan already wrote
    // its vehicle count) and every scenario's clock; no kernel of this step
    // reads them after this point
    if (vb == 0) {
        if (threadIdx.x == 0) {
            c.cnt_next->n_ent = 0;
            c.cnt_next->n_cand = 0;
            c.cnt_next->n_late = 0;
            c.cnt_next->res_done = 0;
            c.cnt_next->ticket_lane = 0;
            c.cnt_next->tag = tag >= 0x3fffffff ? 1 : tag + 1;
        }
        for (int s = threadIdx.x; s < c.n_scen; s += TILE) {
            if (c.scen_ctl[s]) continue;  // frozen or retiring: its clock stands still
            const long long t = c.scen_step[s] + 1;
            c.scen_step[s] = t;
            if (t == c.stop_at[s]) c.scen_ctl[s] = SC_FROZEN;  // reached its horizon
        }
    }
    __shared__ int s_lpre[TILE + 1];  // leavers among the tile's slots before each slot (and in all)
    __shared__ int s_first[2];        // start and end of the lane that holds the tile's first slot
    for (int tile = vb; tile < n_tiles; tile += nvb) {
        const int t0 = tile * TILE;
        const int i = t0 + threadIdx.x;
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
        if (threadIdx.x == 0) {
            s_first[0] = c.cur.off[A.lane];
            s_first[1] = c.cur.off[A.lane + 1];
        }
        __syncthreads();
        int wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += s_warp[w];
        s_lpre[threadIdx.x] = wbase + wpre;
        if (threadIdx.x == TILE - 1) s_lpre[TILE] = wbase + wpre + leaver;
        // a lane that covers the whole tile: its leavers before the tile
        const int f0 = s_first[0], f1 = s_first[1];
        int pre0 = 0;
        if (f0 < t0 && f1 > t0 + TILE)
            for (int k0 = t0; k0 > f0; k0 -= TILE) {
                const int k = k0 - 1 - (int)threadIdx.x;
                pre0 += __syncthreads_count(k >= f0 && c.code[k] != C_STAY);
            }
        __syncthreads();
        if (valid && code == C_STAY) {
            // its rank among the lane's stayers: from the lane's start (slots
            // ahead of it minus the leavers among them) when the lane starts
            // in the tile; from the lane's end (the lane's stayers minus
            // those behind it) when the lane started before the tile and
            // ends in it; else with the leavers before the tile counted above
            const int lane = A.lane;
            const int ob = c.cur.off[lane], oe = c.cur.off[lane + 1];
            const int o0 = c.nxt.off[lane], o1 = c.nxt.off[lane + 1];
            int n_in = 0;
            const int ent = entrants_ahead(c, lane, w.s, A.id, tag, &n_in);
            const int x = threadIdx.x;
            int stay_rank;
            if (ob >= t0) {
                stay_rank = (i - ob) - (s_lpre[x] - s_lpre[ob - t0]);
            } else if (oe <= t0 + TILE) {
                const int behind = (oe - 1 - i) - (s_lpre[oe - t0] - s_lpre[x + 1]);
                stay_rank = (o1 - o0 - n_in) - 1 - behind;
            } else {
                stay_rank = (i - ob) - (pre0 + s_lpre[x]);
            }
            const int pos = o0 + stay_rank + ent;
            if (pos < o0 || pos >= o1) {
                atomicOr(c.err, ERR_RANGE);
            } else {
                RecA<Real> O;
                O.s = w.s; O.v = w.v; O.id = A.id; O.lane = lane;
                c.nxt.a[pos] = O;
                c.nxt.b[pos] = B;
            }
        }
        __syncthreads();  // s_warp, s_lpre and s_first serve the next tile
    }
    // entrants: one warp per entrant.  The stayers of a lane keep their
    // order (nobody overtakes within a lane, R13), so the stayers behind an
    // entrant form the rear of the lane's old segment: the warp counts them
    // from the segment's end, 32 slots per round, and stops at the first
    // round that holds a stayer ahead of the entrant (entrants join mostly
    // at the rear of a lane: one round).  Stayers ahead = the lane's stayers
    // (its next size minus its entrants) minus those behind.
    const int gwarp = vb * (TILE / 32) + warp, nwarps = nvb * (TILE / 32);
    for (int q = gwarp; q < n_ent; q += nwarps) {
        const RecA<Real> Q = c.ea[q];
        const int lane = Q.lane;
        const int b = c.cur.off[lane], e = c.cur.off[lane + 1];
        int behind = 0;
        for (int k0 = e - 1; k0 >= b; k0 -= 32) {
            const int k = k0 - lane_id;
            bool st = false, ah = false;
            if (k >= b && c.code[k] == C_STAY) {
                st = true;
                ah = ahead(c.stay[k].s, c.cur.a[k].id, Q.s, Q.id);
            }
            behind += __popc(__ballot_sync(0xffffffffu, st && !ah));
            if (__any_sync(0xffffffffu, ah)) break;
        }
        if (lane_id == 0) {
            int n_in = 0;
            const int ent_ahead = entrants_ahead(c, lane, Q.s, Q.id, tag, &n_in);
            const int o0 = c.nxt.off[lane], o1 = c.nxt.off[lane + 1];
            const int pos = o0 + (o1 - o0 - n_in - behind) + ent_ahead;
            if (pos < o0 || pos >= o1) {
                atomicOr(c.err, ERR_RANGE);
            } else {
                c.nxt.a[pos] = Q;
                c.nxt.b[pos] = c.eb[q];
            }
        }
    }
    // clear the lane look-back words for the next step (k_lanescan is done)
    for (int k = vb * TILE + threadIdx.x; k < c.n_lane_tiles; k += nvb * TILE)
        c.lane_tiles[k] = 0ull;
}

template <typename Real>
__global__ void __launch_bounds__(TILE) k_place(Ctx<Real> c) {
    if (*c.err & ERR_POISON) return;
    place_blocks(c, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// The whole step as one cooperative launch (every block resident at once):
// the work of k_decide, k_lanescan and k_place as three phases separated by
// grid-wide barriers.  A barrier is a count of arrived blocks and a
// generation word; a wait that exceeds SPIN_LIMIT sets ERR_TIMEOUT and every
// block leaves the step.
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(bar[1]);
        const unsigned g = gen.load(cuda::memory_order_relaxed);
        __threadfence();
        if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
            bar[0] = 0u;
            gen.store(g + 1u, cuda::memory_order_release);
        } else {
            long long spins = 0;
            while (gen.load(cuda::memory_order_acquire) == g) {
                if (++spins > SPIN_LIMIT) { atomicOr(err, ERR_TIMEOUT); break; }
                if (spins > 16) __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = !(*((volatile int*)err) & ERR_POISON);
    }
    __syncthreads();
    return s_ok != 0;
}

#ifndef MOSS_COOP_MIN_BLOCKS
#define MOSS_COOP_MIN_BLOCKS 4
#endif
template <typename Real, bool Groups>
__global__ void __launch_bounds__(TILE, MOSS_COOP_MIN_BLOCKS) k_step_coop(Ctx<Real> c, int n_work, int n_ins,
                                                                          unsigned* bar) {
    if (*c.err & ERR_POISON) return;
    // decide: n_work tile runs, then n_ins insertion blocks, as virtual blocks
    for (int vb = blockIdx.x; vb < n_work + n_ins; vb += gridDim.x)
        decide_block<Real, Groups>(c, n_work, vb, n_work + n_ins);
    if (!grid_sync(bar, c.err)) return;
    lanescan_blocks(c);
    if (!grid_sync(bar, c.err)) return;
    place_blocks(c, blockIdx.x, gridDim.x);
}

// signal states for the current step of every junction (after creation or
// a state reset)
template <typename Real>
__global__ void k_junction_init(Ctx<Real> c, int j0, int j1) {
    for (int j = j0 + blockIdx.x * blockDim.x + threadIdx.x; j < j1; j += gridDim.x * blockDim.x)
        c.junc_state[j] = junction_state_at(c, j, 0);
}

// setter: policy (and manual phase) of n junctions, effective from the
// current step (the state of the step is recomputed)
template <typename Real>
__global__ void k_set_signal(Ctx<Real> c, int n, const int32_t* ids, const int32_t* phases, int policy) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int j = ids[k];
    if (policy == POL_MAXP) {
        // starts, green, the phase the junction shows at this step (R23)
        const int st = c.junc_state[j];
        c.mp[j] = make_int4((st & 512) ? 0 : (st & 15), 1, -1, 0);
    }
    const int was = c.junc_policy[j] == POL_MAXP, now = policy == POL_MAXP;
    if (was != now) atomicAdd(c.n_mp, now - was);
    c.junc_policy[j] = policy;
    if (policy == POL_MANUAL) c.junc_manual[j] = phases[k];
    c.junc_state[j] = junction_state_at(c, j, 0);
}

// lane setters (R25): speed limit (mode 0, value as float bits) or
// restriction flag (mode 1) of n lanes, effective from the next step
template <typename Real>
__global__ void k_set_lane(Ctx<Real> c, int n, const int32_t* ids, const int32_t* vals, int mode) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    LaneInfo* li = const_cast<LaneInfo*>(c.lane) + ids[k];
    if (mode == 0) li->vmax = __int_as_float(vals[k]);
    else li->flags = vals[k] ? (li->flags | LF_RESTRICTED) : (li->flags & ~LF_RESTRICTED);
}

// metrics of the current snapshot (R24): queue length of lanes [l0, l1) —
// vehicles with v < 0.1 m/s within the last 50 m (the lane's segment is
// ordered from its end, so the scan stops at the first vehicle farther away)
template <typename Real>
__global__ void k_lane_queue(Ctx<Real> c, int l0, int l1, int32_t* out) {
    const int l = l0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= l1) return;
    const double L = (double)c.lane[l].L;
    int q = 0;
    for (int k = c.cur.off[l]; k < c.cur.off[l + 1]; ++k) {
        const RecA<Real> a = c.cur.a[k];
        if (L - (double)a.s > 50.0) break;
        if ((double)a.v < 0.1) ++q;
    }
    out[l - l0] = q;
}

// average vehicle speed of roads [r0, r1) (R24): mean speed of the vehicles
// on the road's lanes, the mean speed limit of its lanes when it is empty
template <typename Real>
__global__ void k_road_speed(Ctx<Real> c, int r0, int r1, double* out) {
    const int r = r0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= r1) return;
    const int2 sp = c.road_span[r];
    double sum = 0.0, lim = 0.0;
    int cnt = 0;
    for (int l = sp.x; l < sp.y; ++l) {
        lim += (double)c.lane[l].vmax;
        for (int k = c.cur.off[l]; k < c.cur.off[l + 1]; ++k) sum += (double)c.cur.a[k].v;
        cnt += c.cur.off[l + 1] - c.cur.off[l];
    }
    out[r - r0] = cnt > 0 ? sum / (double)cnt : lim / (double)(sp.y - sp.x);
}

// Re-routing (R26): mark the requested vehicles (req[vid] = their index in
// the request, -1 otherwise), find the lanes of the active ones, and give
// them their new routes (route spans; for the active ones the snapshot
// record's route cursor, last road and next lane).
__global__ void k_mark_vehicles(int32_t* req, int n, const int32_t* vids, int on) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) req[vids[k]] = on ? k : -1;
}

template <typename Real>
__global__ void k_find_lanes(Ctx<Real> c, const int32_t* req, int32_t* lane_out) {
    const int n = c.cnt->n_cur;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const RecA<Real> a = c.cur.a[i];
        const int k = req[a.id];
        if (k >= 0) lane_out[k] = a.lane;
    }
}

template <typename Real>
__global__ void k_apply_routes(Ctx<Real> c, const int32_t* req, int nv, const int32_t* vids, const int2* spans) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nv; k += gridDim.x * blockDim.x)
        const_cast<int2*>(c.route_span)[vids[k]] = spans[k];
    const int n = c.cnt->n_cur;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const RecA<Real> a = c.cur.a[i];
        const int k = req[a.id];
        if (k < 0) continue;
        RecB b = c.cur.b[i];
        b.rptr = spans[k].x;
        b.rlast = spans[k].y - 1;
        const LaneInfo li = c.lane[a.lane];
        if (li.lo >= 0) b.nl = b.rptr < b.rlast ? jl_toward(c, li, c.routes[b.rptr + 1]) : -1;
        c.cur.b[i] = b;
    }
}

// Lane plans (R28): road roads[k] switches to plan plans[k] (junction lanes
// outside it get LF_OFF) and is marked; then the vehicles on the marked
// roads' lanes get their next lane again; then the marks are cleared.
template <typename Real>
__global__ void k_set_plan(Ctx<Real> c, int n, const int32_t* roads, const int32_t* plans, const int32_t* jl_plans,
                           int8_t* road_mark) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int r = roads[k], p = plans[k];
    const int2 sp = c.road_span[r];
    LaneInfo* lanes = const_cast<LaneInfo*>(c.lane);
    for (int l = sp.x; l < sp.y; ++l)
        for (int j = lanes[l].jb; j < lanes[l].je; ++j) {
            const bool on = (jl_plans[j] >> p) & 1;
            lanes[j].flags = on ? (lanes[j].flags & ~LF_OFF) : (lanes[j].flags | LF_OFF);
        }
    road_mark[r] = 1;
}

template <typename Real>
__global__ void k_plan_next_lanes(Ctx<Real> c, const int8_t* road_mark) {
    const int n = c.cnt->n_cur;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const RecA<Real> a = c.cur.a[i];
        const LaneInfo li = c.lane[a.lane];
        if (li.lo < 0 || !road_mark[li.road]) continue;
        RecB b = c.cur.b[i];
        b.nl = b.rptr < b.rlast ? jl_toward(c, li, c.routes[b.rptr + 1]) : -1;
        c.cur.b[i] = b;
    }
}

__global__ void k_unmark_roads(int n, const int32_t* roads, int8_t* road_mark) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) road_mark[roads[k]] = 0;
}

// single values written in stream order (slot control, horizons)
__global__ void k_put_i32(int32_t* p, int32_t v) { *p = v; }
__global__ void k_put_i64(long long* p, long long v) { *p = v; }

// Failure-detection self-test: the look-back of tile 1 waits on tile word 0,
// which nothing publishes, so the bounded wait must give up and report.
__global__ void k_selftest_wait(unsigned long long* words, int* err) {
    bool timeout = false;
    warp_lookback(words, 1, &timeout);
    if (threadIdx.x == 0 && timeout) atomicOr(err, ERR_TIMEOUT);
}

}  // namespace moss
