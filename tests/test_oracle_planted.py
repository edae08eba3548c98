"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check
that the pin battery catches every one of them."""
import os
import subprocess
import sys
import tempfile

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
]

BATTERY = r"""
import sys
sys.path.insert(0, {tests!r}); sys.path.insert(0, {root!r})
import oracle_pins as P
lib = sys.argv[1]
for c in P.ALL_CHECKS + [P.check_permutation_invariance]:
    c(libpath=lib)
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
