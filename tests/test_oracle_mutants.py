"""Planted mistakes in a copy of the oracle. Each mutant changes one thing in one function of
oracle/orc_gmacop.c: a dropped term, a wrong sign, index, constant, shift or comparison. The test compiles
it from a temporary copy (the oracle's own source and library are never touched) and runs the pins of the
part it changes against that library (ORC_LIB). The pins must fail. An unmodified copy built the same way
must pass them, which shows that the harness itself works. No GPU.

Not planted, because each is equivalent to the original and no test can tell them apart:
- `key < best_key` against `key <= best_key` in the best-route rule: keys (T, iteration, ant) are unique;
- dropping the per-iteration queue update of a solve: densities and red times are fixed during a solve,
  so it recomputes the order it already holds.
"""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "orc_gmacop.c")

PRIM, SOLVE, TICK = "test_oracle_primitives.py", "test_oracle_solve.py", "test_oracle_tick.py"
EXACT, FRAC, LIT = "test_oracle_exact_h.py", "test_oracle_frac.py", "test_oracle_literal.py"

# (name, text in the oracle, its replacement, pin modules that must catch it)
MUTANTS = [
    # Philox4x32-10 (known-answer vectors) and the draw's counter layout
    ("philox_multiplier", "M0 = 0xD2511F53u", "M0 = 0xD2511F55u", [PRIM]),
    ("philox_key_schedule", "k1 += W1;", "k1 += W0;", [PRIM]),
    ("philox_word_swap", "uint32_t y0 = hi1 ^ x1 ^ k0;", "uint32_t y0 = hi1 ^ x1 ^ k1;", [PRIM]),
    ("philox_key_bump_first", "if (round > 0) {", "if (round >= 0) {", [PRIM]),
    ("draw_counter_order", "uint32_t c[4] = {it, ant, step, stream};", "uint32_t c[4] = {ant, it, step, stream};",
     [SOLVE]),
    # road attributes and the straight-line bound
    ("isqrt_comparison", "if (n >= root + bit) {", "if (n > root + bit) {", [PRIM]),
    ("free_flow_no_rounding", "(uint64_t)length_dm * 360u + speed_kmh / 2u", "(uint64_t)length_dm * 360u", [PRIM]),
    ("capacity_spacing", "lanes * length_dm / 75u", "lanes * length_dm / 70u", [PRIM]),
    ("edge_time_floor", "uint64_t floor_den = cap / 20u;", "uint64_t floor_den = cap / 10u;", [PRIM]),
    ("edge_time_denominator", "den = cap - n;", "den = cap - n + 1;", [PRIM]),
    ("queue_delay_lanes", "(uint64_t)n * h_sat_ms / lanes;", "(uint64_t)n * h_sat_ms;", [PRIM]),
    ("kappa_speed", "((uint64_t)360u << 16) / v_max_kmh", "((uint64_t)360u << 16) / (v_max_kmh + 1)", [PRIM, SOLVE]),
    ("heuristic_dy_term", "(uint64_t)(dx * dx) + (uint64_t)(dy * dy)", "(uint64_t)(dx * dx) + (uint64_t)(dx * dx)",
     [PRIM, SOLVE]),
    # the preemptive phase order and the signal wait
    ("threshold_fraction", "* 3u / 4u; /* Comp_Thres", "* 2u / 3u; /* Comp_Thres", [PRIM, TICK]),
    ("over_longest_first", "Q[p] > Th[p] && (best < 0 || Q[p] > Q[best])", "Q[p] > Th[p] && (best < 0 || Q[p] < Q[best])",
     [PRIM]),
    ("starvation_not_strict", "if (red_ms[p] > T_max)", "if (red_ms[p] >= T_max)", [PRIM, TICK]),
    ("empty_phases_not_last", "if (!used[p] && Q[p] > 0) {", "if (!used[p]) {", [PRIM]),
    ("starved_shortest_first", "red_ms[p] > T_max && (best < 0 || red_ms[p] > red_ms[best])",
     "red_ms[p] > T_max && (best < 0 || red_ms[p] < red_ms[best])", [PRIM]),
    ("longest_queue_tie_high", "if (Q[p] > 0 && (best < 0 || Q[p] > Q[best]))", "if (Q[p] > 0 && (best < 0 || Q[p] >= Q[best]))",
     [PRIM]),
    ("wait_wraps_wrongly", "return (uint32_t)((start + cycle - c) % cycle);", "return (uint32_t)((start + cycle - c - 1) % cycle);",
     [PRIM]),
    ("green_window_end", "if (c >= start && c < start + green[phase])", "if (c >= start && c <= start + green[phase])",
     [PRIM]),
    ("signal_offset_sign", "(arr_ms % cycle + cycle - (offset % cycle)) % cycle", "(arr_ms % cycle + (offset % cycle)) % cycle",
     [PRIM]),
    # the next-node rule
    ("score_beta_minus_one", "return p * pow_int(eta, beta);", "return p * pow_int(eta, beta ? beta - 1 : 0);",
     [PRIM, SOLVE]),
    ("score_alpha_plus_one", "pow_int(orc_tau_factor(tau, flags), alpha);", "pow_int(orc_tau_factor(tau, flags), alpha + 1);",
     [PRIM, SOLVE]),
    ("weight_scale", "floor(ldexp((double)s[i], 22 - E))", "floor(ldexp((double)s[i], 21 - E))", [PRIM]),
    ("roulette_not_strict", "if (acc > r)", "if (acc >= r)", [PRIM, SOLVE]),
    ("cost_without_heuristic", "int64_t cost = (int64_t)S->tt[e] + w + S->h[v] - S->h[u];",
     "int64_t cost = (int64_t)S->tt[e] + w;", [SOLVE]),
    ("cost_without_current_bound", "+ w + S->h[v] - S->h[u];", "+ w + S->h[v];", [SOLVE]),
    ("cost_bound_of_source", "+ w + S->h[v] - S->h[u];", "+ w + S->h[v] - S->h[q->src];", [SOLVE]),
    ("cost_floor_two", "uint32_t c = cost < 1 ? 1u : (uint32_t)cost;", "uint32_t c = cost < 2 ? 2u : (uint32_t)cost;",
     [SOLVE]),
    ("wait_at_destination", "if (v != q->dst && g->n_phases[v] > 0) {", "if (g->n_phases[v] > 0) {", [SOLVE]),
    ("time_without_wait", "t += (uint64_t)S->tt[e] + S->waitv[pick];", "t += (uint64_t)S->tt[e];", [SOLVE]),
    ("no_visited_rule", "if (!S->visited[g->col[e]])", "if (1)", [SOLVE]),
    ("road_to_itself_a_way_on", "if (!S->visited[g->col[e]])", "if (!S->visited[g->col[e]] || g->col[e] == u)",
     [SOLVE]),
    ("step_cap_early", "if (moves == S->max_steps)", "if (moves + 1 == S->max_steps)", [SOLVE]),
    ("default_step_cap", "uint32_t def_steps = two_n < 4096u ? (uint32_t)two_n : 4096u;",
     "uint32_t def_steps = two_n < 4095u ? (uint32_t)two_n : 4095u;", [SOLVE]),
    ("default_step_cap_one_pass", "uint64_t two_n = 2ull * (N - 1u);", "uint64_t two_n = N - 1u;", [SOLVE]),
    # the step back at a dead end
    ("dead_end_fails_at_once", "if (len == 0) {", "if (1) {", [SOLVE]),
    ("back_keeps_wait_in_time", "t -= (uint64_t)S->tt[e] + S->wait_at[len];", "t -= (uint64_t)S->tt[e];", [SOLVE]),
    ("back_keeps_wait", "W -= S->wait_at[len];", "W -= 0;", [SOLVE]),
    ("back_to_source", "u = len ? g->col[route_edges[len - 1]] : q->src;", "u = q->src;", [SOLVE]),
    ("back_not_a_move", "            moves++;\n            continue;", "            continue;", [SOLVE]),
    ("back_forgets_node", "            len--;\n            uint32_t e = route_edges[len];",
     "            S->visited[u] = 0;\n            len--;\n            uint32_t e = route_edges[len];", [SOLVE]),
    ("draw_keyed_by_depth", "draw64(q->seed, it, ant, moves, 0)", "draw64(q->seed, it, ant, len, 0)", [SOLVE]),
    ("log_moves_as_roads", "res->ant_steps += moves;", "res->ant_steps += steps;", [SOLVE]),
    ("time_cap_halved", "if (t > ORC_T_CAP)", "if (t > ORC_T_CAP / 2)", [SOLVE]),
    ("congested_all_dropped", "if (n_ok > 0 && n_ok < n) {", "if (n_ok < n) {", [SOLVE]),
    ("tie_rule_ant_major", "| ((uint64_t)it * q->n_ants + k);", "| ((uint64_t)k * q->n_iter + it);", [SOLVE]),
    ("beta_fraction_ignored", "*frac = floorf(q->alpha) != q->alpha || floorf(q->beta) != q->beta;",
     "*frac = floorf(q->alpha) != q->alpha;", [FRAC]),
    ("visited_not_marked", "S->visited[u] = 1;\n        S->wait_at[len]", "S->wait_at[len]", [SOLVE]),
    ("draw_words_swapped", "return (uint64_t)o[0] | ((uint64_t)o[1] << 32);", "return (uint64_t)o[1] | ((uint64_t)o[0] << 32);",
     [PRIM, SOLVE]),
    ("best_wait_is_time", "best_W = W;", "best_W = T;", [SOLVE]),
    ("no_score_saturation", "if (p > FLT_MAX)", "if (0)", [LIT]),
    ("weight_floor_dropped", "w[i] = q < 1 ? 1 : q;", "w[i] = q;", [PRIM]),
    ("zero_scores_zero_weights", "            w[i] = 1;", "            w[i] = 0;", [PRIM]),
    ("heuristic_scale_shift", "uint64_t h = (orc_isqrt64(d2) * kappa) >> 16;", "uint64_t h = (orc_isqrt64(d2) * kappa) >> 15;",
     [PRIM]),
    ("frac_cost_plus_one", "float B = beta * orc_log2((float)c_ms);", "float B = beta * orc_log2((float)c_ms + 1.0f);",
     [FRAC]),
    # pheromone: initial value, evaporation, deposits
    ("random_tau_word", "tau[e] = ((uint64_t)1 << 31) + o[0];", "tau[e] = ((uint64_t)1 << 31) + o[1];", [PRIM]),
    ("rho_fix_scale", "ldexp((double)rho, 32)", "ldexp((double)rho, 31)", [PRIM, SOLVE]),
    ("evaporation_shift", "(((unsigned __int128)tau * rho_fix) >> 32)", "(((unsigned __int128)tau * rho_fix) >> 33)",
     [PRIM, SOLVE]),
    ("deposit_numerator", "(uint64_t)(S.h[q->src] > 0 ? S.h[q->src] : 1u) << 32",
     "(uint64_t)(S.h[q->src] > 0 ? S.h[q->src] : 1u) << 31", [SOLVE]),
    ("deposit_denominator", "dep_num / T;", "dep_num / (T + 1);", [SOLVE]),
    ("deposit_before_evaporation", "tau[e] = orc_evaporate(tau[e], rho_fix) + D[e];",
     "tau[e] = orc_evaporate(tau[e] + D[e], rho_fix);", [SOLVE]),
    # the paper-literal variant
    ("repulsive_not_reciprocal", "return (flags & ORC_FLAG_REPULSIVE) ? 1.0f / tf : tf;", "return tf;", [LIT]),
    ("unit_deposit_half", "uint64_t delta = unit ? (uint64_t)1 << 32", "uint64_t delta = unit ? (uint64_t)1 << 31", [LIT]),
    ("evaporate_used_roads", "if (D[e] == 0)", "if (D[e] != 0)", [LIT]),
    # non-integer exponents
    ("log2_constant", "LOG_C7 = 0x1.24924ap-3f", "LOG_C7 = 0x1.249250p-3f", [FRAC]),
    ("exp2_power_split", "int n2 = ni - n1;", "int n2 = ni - n1 + 1;", [FRAC]),
    ("exp2_series_term", "for (int k = 7; k >= 0; --k)", "for (int k = 7; k >= 1; --k)", [FRAC]),
    # exact Calc_Dist
    ("dijkstra_relaxation", "uint64_t nd = dist[u] + tt[e];", "uint64_t nd = dist[u] + tt[e] + 1;", [EXACT]),
    ("dijkstra_heap_order", "if (l < n_heap && hk[l] < hk[m])", "if (l < n_heap && hk[l] > hk[m])", [EXACT]),
    ("dijkstra_no_clamp", "h[v] = dist[v] > ORC_H_CLAMP ? ORC_H_CLAMP : (uint32_t)dist[v];", "h[v] = (uint32_t)dist[v];",
     [EXACT]),
    # serving tick
    ("tick_discharge_clock", "(uint64_t)g->lanes[e] * (t_now + dt) / hsat - (uint64_t)g->lanes[e] * t_now / hsat",
     "(uint64_t)g->lanes[e] * dt / hsat", [TICK]),
    ("tick_split_remainder", "(j < K[u] % d ? 1u : 0u)", "(j + 1 < K[u] % d ? 1u : 0u)", [TICK]),
    ("tick_red_empty_phase", "p == gph[v] || Q[i] == 0)", "p == gph[v])", [TICK]),
    ("tick_red_wraps", "r > 0xFFFFFFFFu - dt ? 0xFFFFFFFFu : r + dt", "r + dt", [TICK]),
    ("tick_arrivals_lost", "veh_out[e] = (uint32_t)(g->vehicles[e] - leave[e] + in);",
     "veh_out[e] = (uint32_t)(g->vehicles[e] - leave[e]);", [TICK]),
    ("tick_green_window_end", "c < start + green[p])", "c <= start + green[p])", [TICK]),
    ("red_time_phase_index", "g->red_ms[(size_t)v * ORC_MAX_PHASES + p]", "g->red_ms[(size_t)v * ORC_MAX_PHASES]",
     [PRIM, TICK]),
    ("wait_window_start", "start += green[order[i]];", "start += green[i];", [PRIM]),
]


def _cflags():
    sys.path.insert(0, ROOT)
    from oracle import build

    return build.CFLAGS


def _run(name, old, new, modules, workdir, cflags):
    """Build the mutant (or the unmodified copy when old is None) and run its pins; returns pytest's code."""
    src = open(SRC).read()
    if old is not None:
        src = src.replace(old, new, 1)
    path = os.path.join(workdir, name + ".c")
    lib = os.path.join(workdir, "lib" + name + ".so")
    with open(path, "w") as f:
        f.write(src)
    subprocess.run([os.environ.get("CC", "gcc"), *cflags, "-o", lib, path, "-lm"], check=True, capture_output=True)
    env = dict(os.environ, ORC_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    cmd += [os.path.join(ROOT, "tests", m) for m in modules]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-400:]


def test_each_mutant_text_occurs_once():
    src = open(SRC).read()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, old, new, _ in MUTANTS:
        assert src.count(old) == 1, name
        assert old != new, name


def test_planted_mistakes_fail_their_pins():
    cflags = _cflags()
    every = sorted({m for *_, mods in MUTANTS for m in mods})
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
            control = ex.submit(_run, "unmodified", None, None, every, tmp, cflags)
            runs = [ex.submit(_run, name, old, new, mods, tmp, cflags) for name, old, new, mods in MUTANTS]
            name, code, out = control.result()
            assert code == 0, f"the unmodified copy must pass every pin module:\n{out}"
            survivors = []
            for f in runs:
                name, code, out = f.result()
                if code != 1:  # 1: tests failed; 0: the mutant survived; other codes: the run broke
                    survivors.append((name, code, out))
    assert not survivors, survivors
