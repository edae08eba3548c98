// Kernels of one simulation step (see moss_device.cuh for the layout).
#pragma once

#include "moss_device.cuh"

namespace moss {

// ---------------------------------------------------------------------------
// k_prepare: one thread per lane and per junction.
//   - junction signal state for step t (fixed time / manual / none, R19);
//   - reset of the per-lane entrant lists and counters of this step;
//   - departure insertion (R18): the head of a start lane's FIFO enters at
//     s = 0, v = 0 when it is due and the snapshot's rearmost vehicle on the
//     lane has s - len >= s0 (or the lane is empty).
//   - clears the look-back tile words of this step.
template <typename Real>
__global__ void __launch_bounds__(PREP_THREADS) k_prepare(Ctx<Real> c) {
    if (c.cnt->err & ERR_POISON) return;  // a failed step leaves the state frozen
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    for (int k = gtid; k < c.n_lane_tiles; k += nthreads) c.lane_tiles[k] = 0ull;
    for (int k = gtid; k < c.max_place_tiles; k += nthreads) c.place_tiles[k] = 0ull;
    for (int j = gtid; j < c.n_junctions; j += nthreads) {
        const int s = c.junc_scen[j];
        const long long t = c.scen_step[s];
        const int p0 = c.junc_phase_off[j], np = c.junc_phase_off[j + 1] - p0;
        const int pol = c.junc_policy[j];
        int st;
        if (pol == POL_NONE || np <= 0) {
            st = 512;
        } else if (pol == POL_MANUAL) {
            st = (c.junc_manual[j] & 15) | ((np & 15) << 4);
        } else {
            long long cyc = 0;
            for (int p = 0; p < np; ++p) cyc += c.phase_green[p0 + p] + c.phase_amber[p0 + p];
            if (cyc <= 0) {
                st = 512;
            } else {
                long long x = (t + c.junc_offset[j]) % cyc;
                if (x < 0) x += cyc;
                st = 0;
                for (int p = 0; p < np; ++p) {
                    const long long g = c.phase_green[p0 + p], a = c.phase_amber[p0 + p];
                    if (x < g + a) {
                        st = p | ((np & 15) << 4) | (x >= g ? 256 : 0);
                        break;
                    }
                    x -= g + a;
                }
            }
        }
        c.junc_state[j] = st;
    }
    for (int l = gtid; l < c.n_lanes; l += nthreads) {
        c.head[l] = -1;
        c.enter[l] = 0;
        c.leave[l] = 0;
    }
    // the counters above must be visible before insertion appends; insertion
    // for lane l is done by the same thread that reset lane l.
    for (int l = gtid; l < c.n_lanes; l += nthreads) {
        const int h = c.q_head[l];
        if (h >= c.q_off[l + 1]) continue;
        const int vid = c.q_ids[h];
        const int sc = c.lane_scen[l];
        const long long t = c.scen_step[sc];
        if ((long long)c.dep[vid] > t) continue;
        const int b = c.cur.off[l], e = c.cur.off[l + 1];
        int fl = F_INSERTED;
        if (e > b) {
            const Real sr = c.cur.s[e - 1];
            const Real g = sr - c.len - c.s0;
            const Real scl = sr > Real(1) ? sr : Real(1);
            if (rabs(g) < c.band * scl) fl |= F_FLAGGED;
            if (!(g >= Real(0))) continue;
        }
        const int q = atomicAdd(&c.cnt->n_ent, 1);
        const int r0 = c.route_off[vid], r1 = c.route_off[vid + 1] - 1;
        int nl = -1;
        if (r0 < r1) {
            nl = jl_toward(c, l, c.routes[r0 + 1]);
            if (nl < 0) atomicOr(&c.cnt->err, ERR_ROUTE);
        }
        c.es[q] = Real(0); c.ev[q] = Real(0); c.elane[q] = l; c.eid[q] = vid;
        c.ev0f[q] = c.v0f[vid]; c.erptr[q] = r0; c.erlast[q] = r1; c.enl[q] = nl;
        c.enext[q] = c.head[l];
        c.head[l] = q;
        c.enter[l] += 1;
        c.q_head[l] = h + 1;
        c.vstatus[vid] = 1;
        c.vflags[vid] = int((t & 0xFFFFFF) << 8) | fl;
        long long* M = c.metrics + (long long)sc * M_NFIELDS;
        atomicAdd((unsigned long long*)&M[M_INSERTED], 1ull);
        atomicAdd((unsigned long long*)&M[M_CUR_ACTIVE], 1ull);
        if (fl & F_FLAGGED) atomicAdd((unsigned long long*)&M[M_FLAGGED], 1ull);
    }
}

// ---------------------------------------------------------------------------
// k_decide: one thread per vehicle of the current snapshot.
template <typename Real>
__global__ void __launch_bounds__(DECIDE_THREADS) k_decide(Ctx<Real> c) {
    if (c.cnt->err & ERR_POISON) return;
    const int n = c.cnt->n_cur;
    const int per_block = (n + gridDim.x - 1) / gridDim.x;
    const int beg = blockIdx.x * per_block;
    const int end = min(n, beg + per_block);
    MetricAcc acc;
    macc_reset(acc, -1);
    for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
        const int lane = c.cur.lane[i];
        const int nl0 = c.cur.nl[i];
        if ((unsigned)lane >= (unsigned)c.n_lanes || nl0 < -1 || nl0 >= c.n_lanes) {
            atomicOr(&c.cnt->err, ERR_RANGE);
            continue;
        }
        const int sc = c.lane_scen[lane];
        if (sc != acc.scen) {
            macc_flush_thread(acc, c.metrics);
            macc_reset(acc, sc);
        }
        const long long t = c.scen_step[sc];
        const uint32_t k0 = c.key0[sc], k1 = c.key1[sc];
        const int vbase = c.veh_base[sc];
        Decision<Real> D = decide(c, i, t, k0, k1, vbase);
        int fl = D.flag ? F_FLAGGED : 0;
        bool granted = false;
        if (D.cand) {
            fl |= F_CANDIDATE;
            granted = true;
            // rivals: candidates of the lane beyond the target lane that fall
            // into the same target-lane gap (TL ahead of them, them ahead of TF)
            const int ol = D.tl + D.dir;  // lane of potential rivals
            const int2 lh = c.lohi[lane];
            if (ol >= lh.x && ol < lh.y) {
                const int ob = c.cur.off[ol], oe = c.cur.off[ol + 1];
                int ra = ob, rb = oe;
                // first slot behind TL, first slot not ahead of TF
                if (D.TL >= 0) ra = partition_point(c, ob, oe, c.cur.s[D.TL], c.cur.id[D.TL]);
                if (D.TF >= 0) rb = partition_point(c, ob, oe, c.cur.s[D.TF], c.cur.id[D.TF]);
                const int my_id = c.cur.id[i];
                for (int r = ra; r < rb; ++r) {
                    const Decision<Real> R = decide(c, r, t, k0, k1, vbase);
                    if (!R.cand || R.tl != D.tl) continue;
                    const Real sc2 = D.scale > R.scale ? D.scale : R.scale;
                    if (rabs(D.u - R.u) < c.band * sc2) fl |= F_FLAGGED;
                    const int rid = c.cur.id[r];
                    const bool win = D.u > R.u || (D.u == R.u && my_id < rid);
                    if (!win) granted = false;
                }
            }
            if (!granted) fl |= F_CONFLICT_LOST;
        }
        // ---- integration (R12, R13)
        const LaneAcc<Real>& la = granted ? D.tgt : D.own;
        int nlane = granted ? D.tl : lane;
        if (granted) fl |= F_CHANGED;
        const Real s = c.cur.s[i], v = c.cur.v[i], a = la.a, dt = c.dt;
        Real vn = v + a * dt, disp;
        if (vn >= Real(0)) {
            disp = v * dt + Real(0.5) * a * dt * dt;
        } else {
            disp = -v * v / (Real(2) * a);
            vn = Real(0);
        }
        if (la.has_leader) { const Real cl = la.gap > Real(0) ? la.gap : Real(0); if (disp > cl) disp = cl; }
        if (la.stop) { const Real cl = la.stop_gap > Real(0) ? la.stop_gap : Real(0); if (disp > cl) disp = cl; }
        Real sn = s + disp;
        if (la.stop && sn > Real(c.L[nlane])) sn = Real(c.L[nlane]);
        // ---- transfer and arrival (R17).  The overshoot past the lane end is
        // taken as disp - (L - s): L - s is exact for s >= L/2 (Sterbenz), so
        // the position on the next lane does not lose the bits of L.
        int rptr = c.cur.rptr[i];
        const int rlast = c.cur.rlast[i];
        int nl = la.nl;
        bool arrived = false;
        Real ex = disp - (Real(c.L[nlane]) - s);  // distance beyond the end of nlane
        for (int iter = 0;; ) {
            const Real Ll = Real(c.L[nlane]);
            const Real scl = Ll > Real(1) ? Ll : Real(1);
            if (la.stop && iter == 0) break;
            const bool road = c.lohi[nlane].x >= 0;
            if (road && rptr == rlast) {
                if (rabs(ex) < c.band * scl) fl |= F_FLAGGED;
                if (ex >= Real(0)) arrived = true;
                break;
            }
            if (rabs(ex) < c.band * scl) fl |= F_FLAGGED;
            if (!(ex > Real(0))) break;
            if (++iter > 4 || nl < 0) { atomicOr(&c.cnt->err, ERR_TRANSFER); sn = Ll; break; }
            sn = ex;
            fl |= F_TRANSFER;
            if (road) {
                nlane = nl;                 // into the junction lane
                nl = c.lohi[nlane].y;       // its target road lane
            } else {
                nlane = nl;                 // onto the next road
                rptr += 1;
                nl = (rptr < rlast) ? jl_toward(c, nlane, c.routes[rptr + 1]) : -1;
                if (rptr < rlast && nl < 0) atomicOr(&c.cnt->err, ERR_ROUTE);
            }
            ex = sn - Real(c.L[nlane]);
        }
        // ---- outputs
        if (arrived) fl |= F_ARRIVED;
        const int id = c.cur.id[i];
        acc.m[0] += 1;
        acc.m[3] += (long long)llrint(double(vn) * SPEED_FX);
        if (fl & F_FLAGGED) acc.m[5] += 1;
        if (fl & F_CHANGED) acc.m[4] += 1;
        if (D.own.overlap) acc.m[6] += 1;
        c.vflags[id] = int((t & 0xFFFFFF) << 8) | fl;
        if (arrived) {
            c.code[i] = C_ARRIVE;
            c.vstatus[id] = 2;
            acc.m[1] += 1;
            acc.m[2] += (t + 1) - (long long)c.dep[id];
            atomicAdd(&c.leave[lane], 1);
            long long* M = c.metrics + (long long)sc * M_NFIELDS;
            atomicAdd((unsigned long long*)&M[M_CUR_ACTIVE], (unsigned long long)(-1ll));
            atomicAdd((unsigned long long*)&M[M_CUR_ARRIVED], 1ull);
        } else if (nlane == lane) {
            c.code[i] = C_STAY;
            c.rs[i] = sn;
            c.rv[i] = vn;
        } else {
            c.code[i] = C_MOVE;
            atomicAdd(&c.leave[lane], 1);
            const int q = atomicAdd(&c.cnt->n_ent, 1);
            c.es[q] = sn; c.ev[q] = vn; c.elane[q] = nlane; c.eid[q] = id;
            c.ev0f[q] = c.cur.v0f[i]; c.erptr[q] = rptr; c.erlast[q] = rlast; c.enl[q] = nl;
            atomicAdd(&c.enter[nlane], 1);
            c.enext[q] = atomicExch(&c.head[nlane], q);
        }
    }
    macc_flush_block<DECIDE_THREADS>(acc, c.metrics);
}

// ---------------------------------------------------------------------------
// k_lanescan: next-snapshot lane offsets.  newsize(l) = size(l) - leave(l) +
// enter(l).  Two exclusive prefix sums (new sizes, leavers) over lanes in one
// decoupled look-back pass; tile words pack (flag:2 | leavers:31 | sizes:31).
template <typename Real>
__global__ void __launch_bounds__(LANESCAN_THREADS) k_lanescan(Ctx<Real> c) {
    if (c.cnt->err & ERR_POISON) return;
    __shared__ int s_tile;
    __shared__ long long s_sum[LANESCAN_THREADS];
    __shared__ unsigned long long s_prefix;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&c.cnt->ticket_lane, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= c.n_lane_tiles) return;
        const int base = tile * LANESCAN_TILE + threadIdx.x * LANESCAN_ITEMS;
        int ns[LANESCAN_ITEMS], lv[LANESCAN_ITEMS];
        long long tn = 0, tl = 0;
#pragma unroll
        for (int k = 0; k < LANESCAN_ITEMS; ++k) {
            const int l = base + k;
            if (l < c.n_lanes) {
                const int sz = c.cur.off[l + 1] - c.cur.off[l];
                lv[k] = c.leave[l];
                ns[k] = sz - lv[k] + c.enter[l];
            } else {
                ns[k] = 0; lv[k] = 0;
            }
            tn += ns[k]; tl += lv[k];
        }
        // block-wide inclusive scan of (tn, tl) packed in one 64-bit value
        long long packed = (tl << 31) | tn;
        s_sum[threadIdx.x] = packed;
        __syncthreads();
        for (int o = 1; o < LANESCAN_THREADS; o <<= 1) {
            const long long x = threadIdx.x >= o ? s_sum[threadIdx.x - o] : 0;
            __syncthreads();
            s_sum[threadIdx.x] += x;
            __syncthreads();
        }
        const long long incl = s_sum[threadIdx.x];
        const long long total = s_sum[LANESCAN_THREADS - 1];
        if (threadIdx.x == 0) {
            unsigned long long prefix = 0;
            unsigned long long* st = c.lane_tiles;
            if (tile == 0) {
                store_release(&st[0], (2ull << 62) | (unsigned long long)total);
            } else {
                store_release(&st[tile], (1ull << 62) | (unsigned long long)total);
                int p = tile - 1;
                long long spins = 0;
                while (p >= 0) {
                    const unsigned long long w = load_acquire(&st[p]);
                    const unsigned long long f = w >> 62;
                    if (f == 0) {
                        if (++spins > SPIN_LIMIT) { atomicOr(&c.cnt->err, ERR_TIMEOUT); break; }
                        if (spins > 64) __nanosleep(100);
                        continue;
                    }
                    prefix += w & ((1ull << 62) - 1);
                    if (f == 2) break;
                    --p;
                }
                store_release(&st[tile], (2ull << 62) | (prefix + (unsigned long long)total));
            }
            s_prefix = prefix;
        }
        __syncthreads();
        const unsigned long long pre = s_prefix;
        long long excl = (long long)pre + incl - packed;
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
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_place: writes the next snapshot.  Tiles [0, n_stay_tiles) cover the
// current slots (vehicles that kept their lane keep their relative order;
// their rank = stayers ahead in the lane + entrants ahead of them); the
// remaining tiles cover the entrants (rank = stayers ahead + entrants ahead).
template <typename Real>
__device__ __forceinline__ int entrants_ahead(const Ctx<Real>& c, int lane, Real s, int id) {
    int cnt = 0, guard = 0;
    for (int q = c.head[lane]; q >= 0; q = c.enext[q]) {
        if (q != -1 && ahead(c.es[q], c.eid[q], s, id)) ++cnt;
        if (++guard > (1 << 24)) { atomicOr(&c.cnt->err, ERR_RANGE); break; }
    }
    return cnt;
}

template <typename Real>
__global__ void __launch_bounds__(PLACE_THREADS) k_place(Ctx<Real> c) {
    if (c.cnt->err & ERR_POISON) return;
    __shared__ int s_tile;
    __shared__ int s_warp[PLACE_THREADS / 32];
    __shared__ unsigned long long s_prefix;
    const int n = c.cnt->n_cur;
    const int n_ent = c.cnt->n_ent;
    const int n_stay_tiles = (n + PLACE_TILE - 1) / PLACE_TILE;
    const int n_ent_tiles = (n_ent + PLACE_TILE - 1) / PLACE_TILE;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&c.cnt->ticket_place, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= n_stay_tiles + n_ent_tiles) break;
        if (tile < n_stay_tiles) {
            const int i = tile * PLACE_TILE + threadIdx.x;
            const bool valid = i < n;
            const int8_t code = valid ? c.code[i] : C_STAY;
            const int leaver = (valid && code != C_STAY) ? 1 : 0;
            // block exclusive scan of leaver flags
            const unsigned ball = __ballot_sync(0xffffffffu, leaver);
            const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
            const int wpre = __popc(ball & ((1u << lane_id) - 1));
            if (lane_id == 0) s_warp[warp] = __popc(ball);
            __syncthreads();
            int wbase = 0, total = 0;
            for (int w = 0; w < PLACE_THREADS / 32; ++w) {
                if (w < warp) wbase += s_warp[w];
                total += s_warp[w];
            }
            if (threadIdx.x == 0) {
                unsigned long long prefix = 0;
                unsigned long long* st = c.place_tiles;
                if (tile == 0) {
                    store_release(&st[0], (2ull << 62) | (unsigned long long)total);
                } else {
                    store_release(&st[tile], (1ull << 62) | (unsigned long long)total);
                    int p = tile - 1;
                    long long spins = 0;
                    while (p >= 0) {
                        const unsigned long long w = load_acquire(&st[p]);
                        const unsigned long long f = w >> 62;
                        if (f == 0) {
                            if (++spins > SPIN_LIMIT) { atomicOr(&c.cnt->err, ERR_TIMEOUT); break; }
                            if (spins > 64) __nanosleep(100);
                            continue;
                        }
                        prefix += w & ((1ull << 62) - 1);
                        if (f == 2) break;
                        --p;
                    }
                    store_release(&st[tile], (2ull << 62) | (prefix + (unsigned long long)total));
                }
                s_prefix = prefix;
            }
            __syncthreads();
            if (valid && code == C_STAY) {
                const long long leavers_before = (long long)s_prefix + wbase + wpre;
                const int lane = c.cur.lane[i];
                const int stay_rank = (i - c.cur.off[lane]) - (int)(leavers_before - c.lbefore[lane]);
                const Real sn = c.rs[i];
                const int id = c.cur.id[i];
                const int pos = c.nxt.off[lane] + stay_rank + entrants_ahead(c, lane, sn, id);
                if (pos < c.nxt.off[lane] || pos >= c.nxt.off[lane + 1]) {
                    atomicOr(&c.cnt->err, ERR_RANGE);
                } else {
                c.nxt.lane[pos] = lane;
                c.nxt.s[pos] = sn;
                c.nxt.v[pos] = c.rv[i];
                c.nxt.id[pos] = id;
                c.nxt.v0f[pos] = c.cur.v0f[i];
                c.nxt.rptr[pos] = c.cur.rptr[i];
                c.nxt.rlast[pos] = c.cur.rlast[i];
                c.nxt.nl[pos] = c.cur.nl[i];
                }
            }
        } else {
            const int q = (tile - n_stay_tiles) * PLACE_TILE + threadIdx.x;
            if (q < n_ent) {
                const int lane = c.elane[q];
                const Real sn = c.es[q];
                const int id = c.eid[q];
                int rank = entrants_ahead(c, lane, sn, id);
                // stayers of this lane ahead of the entrant (old segment of the lane)
                const int b = c.cur.off[lane], e = c.cur.off[lane + 1];
                for (int k = b; k < e; ++k)
                    if (c.code[k] == C_STAY && ahead(c.rs[k], c.cur.id[k], sn, id)) ++rank;
                const int pos = c.nxt.off[lane] + rank;
                if (pos < c.nxt.off[lane] || pos >= c.nxt.off[lane + 1]) {
                    atomicOr(&c.cnt->err, ERR_RANGE);
                } else {
                c.nxt.lane[pos] = lane;
                c.nxt.s[pos] = sn;
                c.nxt.v[pos] = c.ev[q];
                c.nxt.id[pos] = id;
                c.nxt.v0f[pos] = c.ev0f[q];
                c.nxt.rptr[pos] = c.erptr[q];
                c.nxt.rlast[pos] = c.erlast[q];
                c.nxt.nl[pos] = c.enl[q];
                }
            }
        }
        __syncthreads();
    }
    // the last block to finish closes the step: publish the next snapshot
    // size, reset the step counters and advance every scenario's clock
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(&c.cnt->done_place, 1);
        if (done == (int)gridDim.x - 1) {
            __threadfence();
            c.cnt->n_cur = c.cnt->n_next;
            c.cnt->n_ent = 0;
            c.cnt->ticket_lane = 0;
            c.cnt->ticket_place = 0;
            c.cnt->done_place = 0;
            for (int s = 0; s < c.n_scen; ++s) c.scen_step[s] += 1;
            __threadfence();
        }
    }
}

}  // namespace moss
