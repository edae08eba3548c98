"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check
that the pin battery catches every one of them."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "moss_oracle.c")

# (name, original text, planted text)
MUTATIONS = [
    ("idm_dv_sign", "double dyn = v * O->T + v * dv /", "double dyn = v * O->T - v * dv /"),
    ("idm_delta_2", "return O->a_max * (1.0 - r2 * r2 - q * q);", "return O->a_max * (1.0 - r2 - q * q);"),
    ("free_delta_2", "return O->a_max * (1.0 - r2 * r2);", "return O->a_max * (1.0 - r2);"),
    ("gap_without_length", "double gap = S->s[ld] - O->len - s;", "double gap = S->s[ld] - s;"),
    ("mobil_tilde_reversed", "u[side] = (at_ego - D.own.a)", "u[side] = (D.own.a - at_ego)"),
    ("mobil_no_threshold", "(D.at_old - D.a_old)) - O->a_th;", "(D.at_old - D.a_old));"),
    ("mobil_old_terms_swapped", "D.a_old = acc_pair(O, S, OF, lane, vid, s, v);",
     "D.a_old = acc_pair(O, S, OF, lane, -1, 0.0, 0.0);"),
    ("leader_farthest", "if (best < 0 || ahead_of(S, best, S->s[m], m)) best = m;\n    }\n    return best;\n}\n\n/* nearest vehicle behind",
     "if (best < 0 || ahead_of(S, m, S->s[best], best)) best = m;\n    }\n    return best;\n}\n\n/* nearest vehicle behind"),
    ("p_lc_literal_branch", "return O->p_lo + (O->p_hi - O->p_lo) * uT;", "return (O->p_hi - O->p_lo) * uT;"),
    ("amber_as_green", "return ((mask >> nxt) & 1) ? LIGHT_GREEN : LIGHT_AMBER;", "return LIGHT_GREEN;"),
    ("no_stop_line", "S->light[nl1] != LIGHT_GREEN) ||", "S->light[nl1] == LIGHT_RED && 0) ||"),
    ("snapshot_written_in_place", "O->lane[i] = lane; O->s[i] = s_new; O->v[i] = v_new; O->rc[i] = rc;",
     "O->lane[i] = lane; O->s[i] = s_new; O->v[i] = v_new; O->rc[i] = rc; S.s[i] = s_new;"),
    ("insertion_ignores_gap", "ok = g >= 0.0;", "ok = 1;"),
    ("transfer_keeps_offset", "s_new -= Ll;\n", "\n"),
    ("conflict_smaller_wins", "return Dx->u > Dy->u ||", "return Dx->u < Dy->u ||"),
    ("ballistic_euler_position", "disp = v * dt + 0.5 * a * dt * dt;", "disp = v * dt;"),
    ("maxp_pressure_sign", "long d = (long)lane_cnt[O->jl_from[jl]] - (long)lane_cnt[O->jl_target[jl]];",
     "long d = (long)lane_cnt[O->jl_target[jl]] - (long)lane_cnt[O->jl_from[jl]];"),
    ("maxp_upstream_only", "long d = (long)lane_cnt[O->jl_from[jl]] - (long)lane_cnt[O->jl_target[jl]];",
     "long d = (long)lane_cnt[O->jl_from[jl]];"),
    ("maxp_no_amber", "if (O->phase_amber[p0 + p] > 0) { q = best; e = 1; }", "if (0) { q = best; e = 1; }"),
    ("maxp_min_green_off_by_one", "} else if (e >= O->phase_green[p0 + p]) {", "} else if (e > O->phase_green[p0 + p]) {"),
    ("queue_window_100m", "if (O->v[i] < 0.1 && O->L[l] - O->s[i] <= 50.0) out[l]++;",
     "if (O->v[i] < 0.1 && O->L[l] - O->s[i] <= 100.0) out[l]++;"),
    ("restriction_no_stop", "(nl1 >= 0 && O->restricted[nl1]) ||", "(0) ||"),
    ("restriction_ignored_by_mobil", "if (tl < lo || tl >= hi || O->restricted[tl]) continue;",
     "if (tl < lo || tl >= hi) continue;"),
    ("max_speed_setter_ignored", "for (int k = 0; k < n; ++k) O->vmax[lanes[k]] = vmax[k];", "(void)vmax;"),
    ("reroute_drops_road_just_left", "    if (prev >= 0) O->routes[beg + len++] = prev;\n", "\n"),
    ("reroute_start_unchecked", "        if (roads[0] != O->lane_road[O->lane[vid]]) return -1;\n", "\n"),
    ("groups_mobil_may_leave", "        if (next_road >= 0 && !has_access(O, tl, next_road)) continue;  /* leaves the group (R27) */\n",
     "\n"),
    ("groups_no_access_no_stop", " || (lane < O->n_road_lanes && nl1 == -2)) {", ") {"),
    ("groups_mandatory_wrong_way", "int dir = best < lane ? -1 : +1, tl = lane + dir;",
     "int dir = best < lane ? +1 : -1, tl = lane + dir;\n        if (tl < lo || tl >= hi) return D;"),
    ("plans_ignored", "return (O->jl_plans[j] >> O->road_plan[O->lane_road[O->jl_from[j]]]) & 1;", "return 1;"),
    ("maxp_ties_to_smallest", "if (pk > pb || (pk == pb && best != p && k < best)) best = k;",
     "if (pk > pb || (pk == pb && k < best)) best = k;"),
    ("lookahead_frontmost",
     "if (best < 0 || ahead_of(S, best, S->s[m], m)) best = m;\n    }\n    return best;\n}\n\n/* next lane on",
     "if (best < 0 || ahead_of(S, m, S->s[best], best)) best = m;\n    }\n    return best;\n}\n\n/* next lane on"),
    ("lookahead_second_lane_length_dropped", "base += O->L[nl];", ";"),
    ("lookahead_gap_without_length", "double gap = base + S->s[rr] - O->len;", "double gap = base + S->s[rr];"),
    ("lookahead_one_lane", "for (int k = 0; k < 2 && nl >= 0; ++k) {", "for (int k = 0; k < 1 && nl >= 0; ++k) {"),
    ("lookahead_third_lane", "nl = (k == 0) ? next_lane(O, vid, nl, rcn, &rcm) : -1;",
     "nl = next_lane(O, vid, nl, rcn, &rcm);\n            if (k == 1 && nl >= 0) { int rr2 = rearmost_on(S, nl); if (rr2 >= 0) "
     "{ a = idm(O, v, v0, base + O->L[nl] + S->s[rr2] - O->len, v - S->v[rr2]); r.has_leader = 1; r.leader = rr2; } }"),
    ("mobil_side_swapped", "side = q > 0.0 ? 0 : 1;", "side = q > 0.0 ? 1 : 0;"),
    ("mobil_uniform_side_flipped", "if (feas[0] && feas[1]) side = D.u_dir < 0.5 ? 0 : 1;",
     "if (feas[0] && feas[1]) side = D.u_dir < 0.5 ? 1 : 0;"),
    ("mobil_uniform_side_ignores_feasibility", "if (feas[0] && feas[1]) side = D.u_dir < 0.5 ? 0 : 1;",
     "if (1) side = D.u_dir < 0.5 ? 0 : 1;"),
    ("mobil_attempt_gate_not_strict", "if (!(D.u_att < O->p_att)) return D;", "if (!(D.u_att <= O->p_att)) return D;"),
    ("mobil_change_gate_not_strict", "if (!(D.u_lc < D.pLC)) return D;", "if (!(D.u_lc <= D.pLC)) return D;"),
    ("mobil_draw_words_swapped", "D.u_att = unit24(w[0]); D.u_lc = unit24(w[1]);",
     "D.u_att = unit24(w[1]); D.u_lc = unit24(w[0]);"),
    ("philox_counter_order_swapped", "uint32_t ctr[4] = {(uint32_t)vid, (uint32_t)t, 0u, 0u}",
     "uint32_t ctr[4] = {(uint32_t)t, (uint32_t)vid, 0u, 0u}"),
]

# Every check runs; each failed assertion is reported at once (a planted
# mistake may also corrupt the oracle's memory later in the battery, so a
# crash alone does not count as caught).
BATTERY = r"""
import sys
sys.path.insert(0, {tests!r}); sys.path.insert(0, {root!r})
import oracle_pins as P
lib = sys.argv[1]
failed = 0
for c in P.ALL_CHECKS + [P.check_permutation_invariance]:
    try:
        c(libpath=lib)
    except AssertionError:
        failed += 1
        print("FAIL", c.__name__, flush=True)
if not failed:
    print("ALL PINS PASSED")
"""


@pytest.mark.parametrize("name,orig,planted", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, orig, planted, tmp_path):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation anchor for {name} not unique/found"
    bad = src.replace(orig, planted)
    csrc = tmp_path / "bad.c"
    csrc.write_text(bad)
    so = tmp_path / "bad.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(csrc), "-lm"])
    code = BATTERY.format(tests=HERE, root=os.path.dirname(HERE))
    r = subprocess.run([sys.executable, "-c", code, str(so)], capture_output=True, text=True,
                       timeout=600)
    assert "ALL PINS PASSED" not in r.stdout, f"planted mistake {name} was not caught"
    assert "FAIL " in r.stdout, f"planted mistake {name} failed no pin (stderr: {r.stderr[-300:]})"
