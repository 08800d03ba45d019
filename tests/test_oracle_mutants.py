"""The pins catch plausible mistakes planted in the oracle (CPU only).

Each case copies the oracle's C source, plants one mistake, builds the copy
and runs a pin file against it in a child process (``NAVIX_ORACLE_SO``); the
pins must fail.  The draw-to-placement misreadings go against
tests/test_oracle_draw_pins.py, the rule mistakes against the step-by-step
comparisons with the independent rule model and the view mistakes against
the independent window-and-rotate view model (both in
tests/test_oracle_model.py), and the time, reward and cost mistakes against
the hand-worked pins and the cost pins (tests/test_oracle_pins.py,
tests/test_oracle_families.py), and the observation and policy mistakes
against the RGB, full-view and policy pins (tests/test_oracle_model.py,
tests/test_oracle_policy.py).
The unmodified copy must pass each, so a failure is the planted mistake's and
not the mechanism's.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "navix_oracle.c")

MUTANTS = {
    # reading R18 read as "columns outer": the k-th free cell scanned x first
    "free_cells_column_major": [(
        "    for (int y = y0; y <= y1; y++)\n        for (int x = x0; x <= x1; x++) {\n"
        "            if (!is_empty_cell(e, x, y) || (x == skip_x && y == skip_y)) continue;",
        "    for (int x = x0; x <= x1; x++)\n        for (int y = y0; y <= y1; y++) {\n"
        "            if (!is_empty_cell(e, x, y) || (x == skip_x && y == skip_y)) continue;")],
    # reading R12 read as simultaneous moves: every ball sees the grid of the step's start
    "balls_move_on_a_snapshot": [
        ("static void move_balls(orc_env* e)\n{\n", "static void move_balls(orc_env* e)\n{\n    orc_env snap = *e;\n"),
        ("                if (!is_empty_cell(e, x, y)) continue;", "                if (!is_empty_cell(&snap, x, y)) continue;")],
    # reading R12's candidate order read column first (dx outer)
    "ball_candidates_dx_outer": [(
        "        for (int dy = -1; dy <= 1; dy++)\n            for (int dx = -1; dx <= 1; dx++) {",
        "        for (int dx = -1; dx <= 1; dx++)\n            for (int dy = -1; dy <= 1; dy++) {")],
    # LavaGap's gap drawn over one row fewer (the last interior row never open)
    "lavagap_gap_range": [(
        "int gap = 1 + (int)orc_bounded(layout_draw(e, 1), (uint32_t)(S - 2));",
        "int gap = 1 + (int)orc_bounded(layout_draw(e, 1), (uint32_t)(S - 3));")],
    # GoToDoor's colours by a full shuffle step (any of the six each time)
    "gotodoor_colour_shuffle": [(
        "int j = i + (int)orc_bounded(layout_draw(e, k++), (uint32_t)(6 - i));",
        "int j = (int)orc_bounded(layout_draw(e, k++), 6u);")],
    # the crossing order shuffled with one position too few at each step
    "crossing_order_shuffle": [(
        "int j = (int)orc_bounded(layout_draw(e, k++), (uint32_t)(i + 1));",
        "int j = (int)orc_bounded(layout_draw(e, k++), (uint32_t)i);")],
    # KeyCorridor's key and goal cells drawn in the other order
    "keycorridor_key_before_goal": [
        ("    int gx0 = gside == 0 ? 1 : xr + 1, gy0 = grow * (s - 1) + 1;",
         "    uint32_t kg = k++;\n    int gx0 = gside == 0 ? 1 : xr + 1, gy0 = grow * (s - 1) + 1;"),
        ("    kth_free(e, (int)orc_bounded(layout_draw(e, k++), (uint32_t)n), gx0, gx0 + s - 3, gy0, gy0 + s - 3, -1, -1, &gx, &gy);",
         "    kth_free(e, (int)orc_bounded(layout_draw(e, k++), (uint32_t)n), gx0, gx0 + s - 3, gy0, gy0 + s - 3, -1, -1, &gx, &gy);\n    (void)kg;"),
        ("    kth_free(e, (int)orc_bounded(layout_draw(e, k++), (uint32_t)n), kx0, kx0 + s - 3, ky0, ky0 + s - 3, -1, -1, &kx, &ky);",
         "    kth_free(e, (int)orc_bounded(layout_draw(e, kg), (uint32_t)n), kx0, kx0 + s - 3, ky0, ky0 + s - 3, -1, -1, &kx, &ky);")],
    # reading R1's random-action counter with the episode word 0 instead of all ones
    "action_counter_episode_word": [(
        "orc_draw(e->seed, e->env_index, 0xFFFFFFFFu, gstep, PURPOSE_ACTION, 0)",
        "orc_draw(e->seed, e->env_index, 0u, gstep, PURPOSE_ACTION, 0)")],
}


def _build(tmp_path, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, f"mutation site not found exactly once: {old[:60]!r}"
        src = src.replace(old, new)
    c = tmp_path / "navix_oracle.c"
    c.write_text(src)
    so = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I",
                    os.path.join(ROOT, "oracle"), "-o", str(so), str(c)], check=True)
    return str(so)


def _run_pins(so):
    env = dict(os.environ, NAVIX_ORACLE_SO=so)
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_draw_pins.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes_the_pins(tmp_path):
    r = _run_pins(_build(tmp_path, []))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_the_planted_mistake(tmp_path, name):
    r = _run_pins(_build(tmp_path, MUTANTS[name]))
    assert r.returncode != 0, f"the pins did not catch {name}"
    assert "failed" in r.stdout, r.stdout[-2000:]


# Plausible mistakes in the intervention rules (Table 3, Appendix A), each of
# which the step-by-step comparison with the independent rule model must catch.
RULE_MUTANTS = {
    # a locked door opened by a key of any colour
    "unlock_any_colour": [(
        "if (e->carry_ent == ORC_KEY && e->carry_col == fcol) orc_set_cell(e, fx, fy, ORC_DOOR, fcol, ORC_OPEN);",
        "if (e->carry_ent == ORC_KEY) orc_set_cell(e, fx, fy, ORC_DOOR, fcol, ORC_OPEN);")],
    # an open door toggled stays open
    "open_door_does_not_close": [(
        "                    orc_set_cell(e, fx, fy, ORC_DOOR, fcol, ORC_CLOSED);",
        "                    orc_set_cell(e, fx, fy, ORC_DOOR, fcol, ORC_OPEN);")],
    # the carried object dropped onto any walkable cell, not only an empty one
    "drop_onto_walkable": [(
        "if (e->carry_ent != 0 && is_empty_cell(e, fx, fy)) {",
        "if (e->carry_ent != 0 && walkable(fent, fst) && fent != ORC_GOAL && fent != ORC_LAVA) {")],
    # pickup with a full hand swaps nothing but picks again
    "pickup_with_full_hand": [(
        "if (e->carry_ent == 0 && (fent == ORC_KEY || fent == ORC_BALL)) {",
        "if (fent == ORC_KEY || fent == ORC_BALL) {")],
    # GoToDoor's done at a door of any colour
    "done_at_any_door": [(
        "if (e->family == ORC_GOTODOOR && fent == ORC_DOOR && fcol == e->mission) goal = 1;",
        "if (e->family == ORC_GOTODOOR && fent == ORC_DOOR) goal = 1;")],
    # a closed (unlocked) door walked through like an open one
    "walk_through_closed_door": [(
        "    if (ent == ORC_DOOR && st == ORC_OPEN) return 1;",
        "    if (ent == ORC_DOOR && st != ORC_LOCKED) return 1;")],
    # the picked-up object left in its cell
    "pickup_leaves_the_object": [(
        "                set_empty(e, fx, fy);\n",
        "")],
    # stepping onto lava not ending the episode
    "lava_not_terminal": [(
        "                if (fent == ORC_LAVA) lava = 1;\n",
        "")],
    # turning the wrong way for left
    "left_turns_right": [(
        "            e->dir = (e->dir + 3) % 4;\n        } else if (action == ORC_RIGHT) {",
        "            e->dir = (e->dir + 1) % 4;\n        } else if (action == ORC_RIGHT) {")],
}


def _run_rule_pin(so):
    env = dict(os.environ, NAVIX_ORACLE_SO=so)
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_model.py"), "-k", "independent_rule_model"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes_the_rule_pin(tmp_path):
    r = _run_rule_pin(_build(tmp_path, []))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(RULE_MUTANTS))
def test_rule_pin_catches_the_planted_mistake(tmp_path, name):
    r = _run_rule_pin(_build(tmp_path, RULE_MUTANTS[name]))
    assert r.returncode != 0, f"the rule pin did not catch {name}"
    assert "failed" in r.stdout, r.stdout[-2000:]


# Plausible mistakes in the view and its occlusion (Table 4), each of which the
# comparisons with the independent window-and-rotate view model must catch.
VIEW_MUTANTS = {
    # closed doors seen through like open ones
    "closed_doors_transparent": [(
        "    if (ent == ORC_DOOR && st != ORC_OPEN) return 0;",
        "    if (ent == ORC_DOOR && st == ORC_LOCKED) return 0;")],
    # light not spreading diagonally ahead to the right
    "no_diagonal_right": [(
        "                vis[j - 1][i + 1] = 1;\n",
        "")],
    # the rightward sweep only (cells left of a blocked one never lit)
    "no_leftward_sweep": [(
        "            vis[j][i - 1] = 1;\n",
        "")],
    # the right-hand direction taken as the left-hand one (a mirrored view)
    "mirrored_view": [(
        "    int F = e->dir, Rt = (e->dir + 1) % 4;",
        "    int F = e->dir, Rt = (e->dir + 3) % 4;")],
}


def _run_view_pin(so):
    env = dict(os.environ, NAVIX_ORACLE_SO=so)
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_model.py"), "-k", "window_model"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes_the_view_pins(tmp_path):
    r = _run_view_pin(_build(tmp_path, []))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(VIEW_MUTANTS))
def test_view_pins_catch_the_planted_mistake(tmp_path, name):
    r = _run_view_pin(_build(tmp_path, VIEW_MUTANTS[name]))
    assert r.returncode != 0, f"the view pins did not catch {name}"
    assert "failed" in r.stdout, r.stdout[-2000:]


# Plausible mistakes in time, reward and termination (Tables 5, 6, Eq. 1),
# each of which the hand-worked pins and the cost pins must catch.
REWARD_MUTANTS = {
    # Eq. 1 evaluated with the step count before the step
    "eq1_step_before_increment": [(
        "r = e->reward_mode == ORC_REWARD_MINIGRID ? minigrid_goal_reward(e->t, e->max_steps) : 1.0f;",
        "r = e->reward_mode == ORC_REWARD_MINIGRID ? minigrid_goal_reward(e->t - 1, e->max_steps) : 1.0f;")],
    # truncation one step late
    "truncation_one_late": [(
        "    int trunc = e->t >= e->max_steps;",
        "    int trunc = e->t > e->max_steps;")],
    # action_cost charged for done too
    "action_cost_on_done": [(
        "    if (action >= 0 && action < ORC_DONE) r = r - e->action_cost;",
        "    if (action >= 0 && action <= ORC_DONE) r = r - e->action_cost;")],
    # time_cost not charged
    "no_time_cost": [(
        "    r = r - e->time_cost;\n",
        "")],
    # Dynamic-Obstacles with all seven actions instead of three
    "dynobs_seven_actions": [(
        "    int n_act = e->family == ORC_DYNOBS ? 3 : 7;\n    if (action < 0 || action > ORC_DONE) {",
        "    int n_act = 7;\n    if (action < 0 || action > ORC_DONE) {")],
    # a collision with a ball not penalised
    "collision_not_penalised": [(
        "        r = -1.0f;\n        term = 1;",
        "        r = 0.0f;\n        term = 1;")],
    # lava ends the episode with the goal reward
    "lava_pays_the_goal_reward": [(
        "        r = e->lava_reward;",
        "        r = 1.0f;")],
}


def _run_reward_pins(so):
    env = dict(os.environ, NAVIX_ORACLE_SO=so)
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                           os.path.join(ROOT, "tests", "test_oracle_families.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes_the_reward_pins(tmp_path):
    r = _run_reward_pins(_build(tmp_path, []))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(REWARD_MUTANTS))
def test_reward_pins_catch_the_planted_mistake(tmp_path, name):
    r = _run_reward_pins(_build(tmp_path, REWARD_MUTANTS[name]))
    assert r.returncode != 0, f"the reward pins did not catch {name}"
    assert "failed" in r.stdout, r.stdout[-2000:]


# Plausible mistakes in the other observations (Table 4) and in the fused
# policy (reading P1), each caught by the model and policy pins.
OBS_POLICY_MUTANTS = {
    # the agent's own tile in the egocentric RGB view not marked
    "rgb_agent_tile_unmarked": [(
        "    if (agent_cell) t += 198;\n",
        "")],
    # the fully observable view showing what lies under the agent
    "full_view_hides_no_agent": [(
        "            } else if (x == e->ax && y == e->ay) {\n                o[0] = ORC_AGENT;",
        "            } else if (0) {\n                o[0] = ORC_AGENT;")],
    # the policy's hidden units not clamped from above
    "policy_no_upper_clamp": [(
        "static int64_t clamp255(int64_t v) { return v < 0 ? 0 : (v > 255 ? 255 : v); }",
        "static int64_t clamp255(int64_t v) { return v < 0 ? 0 : v; }")],
    # the policy's ties going to the last largest logit
    "policy_last_max": [(
        "        if (a == 0 || z > best_z) {",
        "        if (a == 0 || z >= best_z) {")],
    # the second hidden layer requantised with the first layer's shift
    "policy_layer2_shift1": [(
        "        h2[j] = clamp255(floor_shift(acc, p->shift2));",
        "        h2[j] = clamp255(floor_shift(acc, p->shift1));")],
}


def _run_obs_policy_pins(so):
    env = dict(os.environ, NAVIX_ORACLE_SO=so)
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_model.py"),
                           os.path.join(ROOT, "tests", "test_oracle_policy.py"), "-k",
                           "rgb or full or policy or greedy or shift or tie or wall or hand or exploration or agent"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes_the_observation_and_policy_pins(tmp_path):
    r = _run_obs_policy_pins(_build(tmp_path, []))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(OBS_POLICY_MUTANTS))
def test_observation_and_policy_pins_catch_the_planted_mistake(tmp_path, name):
    r = _run_obs_policy_pins(_build(tmp_path, OBS_POLICY_MUTANTS[name]))
    assert r.returncode != 0, f"the observation and policy pins did not catch {name}"
    assert "failed" in r.stdout, r.stdout[-2000:]
