"""Planted mistakes in a copy of the oracle (CPU only): each plausible slip
-- a wrong tie-break, a misread rule, a dropped term, an off-by-one key --
must make at least one pin in tests/oracle_pins.py fail.  The mistakes are
planted by editing a temporary copy of the C source; the real oracle is
never modified."""
import json
import os
import subprocess
import sys

import pytest

import oracle

TESTS = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(TESTS)

# Runs the pins against one compiled copy in a child process, so a planted
# mistake that corrupts memory (e.g. reporting more bins than there is room
# for) is reported as a crash instead of taking the test session down.
_RUNNER = (
    "import json, sys; sys.path[:0] = [%r, %r]\n"
    "import oracle, oracle_pins as P\n"
    "print(json.dumps(P.failing_pins(oracle.OracleLib(sys.argv[1]))))\n"
) % (ROOT, TESTS)


def failing_pins_isolated(path):
    r = subprocess.run([sys.executable, "-c", _RUNNER, path], capture_output=True, text=True,
                       timeout=600)
    if r.returncode != 0:
        return [f"crashed(rc={r.returncode})"]
    return json.loads(r.stdout.strip().splitlines()[-1])

MUTANTS = {
    "bf_tie_highest_index": ("(c == OR_BF && res < chosen_res)", "(c == OR_BF && res <= chosen_res)"),
    "wf_tie_highest_index": ("(c == OR_WF && res > chosen_res)", "(c == OR_WF && res >= chosen_res)"),
    "fit_strict": ("if (res < w)\n                continue;", "if (res <= w)\n                continue;"),
    "rule5_floor_half": ("if (2 * before < cap && cap <= 2 * after) {",
                         "if (before < cap / 2 && cap / 2 <= after) {"),
    "rule5_dropped": ("if (2 * before < cap && cap <= 2 * after) {", "if (0) {"),
    "rule5_wrong_type": ("bins[nb].type = bins[chosen].type;", "bins[nb].type = 0;"),
    "fallback_largest_type": ("if (B[i] >= w)\n                    t = i;", "if (B[i] >= w)\n                    t = 0;"),
    "used_counts_empty_bins": ("if (bins[x].load > 0) {", "if (bins[x].load >= 0) {"),
    "h2_tie_last_rank": ("if (best_total < 0 || cap_sum < best_total) {",
                         "if (best_total < 0 || cap_sum <= best_total) {"),
    "h2_assignment_not_permuted": ("best_item_bin[perm[q]] = dense[raw[q]];",
                                   "best_item_bin[q] = dense[raw[q]];"),
    "sublist_offset_dropped": ("bin_of_item[a + q] = (int32_t)(bin_offset + dense[raw[q]]);",
                               "bin_of_item[a + q] = (int32_t)(dense[raw[q]]);"),
    "random_key_off_by_one": ("or_random_criterion(seed, (uint64_t)(a + q))",
                              "or_random_criterion(seed, (uint64_t)(a + q + 1))"),
    "splitmix_constant_typo": ("0xBF58476D1CE4E5B9ull", "0xBF58476D1CE4E5B8ull"),
    "preopen_reversed": ("bins[nb].type = i;\n            ++nb;", "bins[nb].type = n - 1 - i;\n            ++nb;"),
    "too_big_against_smallest": ("if (w[j] > B[0])", "if (w[j] > B[n - 1])"),
    "opt_largest_capacity": ("for (int32_t i = n - 1; i >= 0; --i) {  /* smallest capacity first */",
                             "for (int32_t i = 0; i < n; ++i) {"),
    "total_counts_loads": ("sum += B[bins[x].type];", "sum += bins[x].load;"),
    "fit_tests_off_by_one": ("or_fit_tests += (uint64_t)nb;", "or_fit_tests += (uint64_t)nb + 1;"),
    "ff_last_fitting": ('            if (chosen < 0 ||\n                (c == OR_BF && res < chosen_res) ||\n                (c == OR_WF && res > chosen_res)) {\n                chosen = x;\n                chosen_res = res;\n            }\n            if (c == OR_FF)\n                break;\n',
                        '            if (chosen < 0 || c == OR_FF ||\n                (c == OR_BF && res < chosen_res) ||\n                (c == OR_WF && res > chosen_res)) {\n                chosen = x;\n                chosen_res = res;\n            }\n'),
    "rule5_every_item_past_half": ("if (2 * before < cap && cap <= 2 * after) {", "if (cap <= 2 * after) {"),
    "fallback_strict_capacity": ("if (B[i] >= w)\n                    t = i;",
                                 "if (B[i] > w)\n                    t = i;"),
    "permutations_suffix_not_reversed": ("    for (int32_t a = i + 1, b = k - 1; a < b; ++a, --b) {\n        t = p[a]; p[a] = p[b]; p[b] = t;\n    }\n",
                                         ""),
    "random_criterion_mapping": ("return (int32_t)(oracle_splitmix64(seed, key) % 3u);",
                                 "return (int32_t)((oracle_splitmix64(seed, key) >> 1) % 3u);"),
    "zero_weight_accepted": ("if (w[j] < 1)\n            return OR_EINVAL;", "if (w[j] < 0)\n            return OR_EINVAL;"),
    "equal_capacities_accepted": ("if (i > 0 && B[i] >= B[i - 1])", "if (i > 0 && B[i] > B[i - 1])"),
    "h2_types_of_last_permutation": ("                    best_used = used;\n", "                    best_used = used;\n                }\n                {\n"),
    "rule5_strictly_past_half": ("if (2 * before < cap && cap <= 2 * after) {", "if (2 * before < cap && cap < 2 * after) {"),
    "preopen_all_largest_type": ("bins[nb].type = i;\n            ++nb;", "bins[nb].type = 0;\n            ++nb;"),
    "h2_preopen_ignored": ("                const int64_t nb = or_membrane_run(seq, crit, k, B, n, preopen, bins, raw, remark3);\n                int64_t cap_sum = 0;\n                const int64_t used = or_used_bins(bins, nb, B, dense, &cap_sum);\n                if (best_total",
                           "                const int64_t nb = or_membrane_run(seq, crit, k, B, n, 0, bins, raw, remark3);\n                int64_t cap_sum = 0;\n                const int64_t used = or_used_bins(bins, nb, B, dense, &cap_sum);\n                if (best_total"),
    "h2_sublist_offset_dropped": ("            bin_offset += best_used;", "            bin_offset += 0;"),
    "remark3_condition_ignored": ("if (!remark3 || or_type_all_half(bins, nb, B, bins[chosen].type)) {",
                                  "if (1) {"),
    "remark3_below_half_strict": ("if (bins[x].type == t && 2 * bins[x].load < (int64_t)B[t])",
                                  "if (bins[x].type == t && 2 * bins[x].load < (int64_t)B[t] - 1)"),
    "h2_random_key_720_as_120": ("? (uint64_t)((g * 720 + rank) * 8 + q)", "? (uint64_t)((g * 120 + rank) * 8 + q)"),
    "h2_random_key_stride_7": ("? (uint64_t)((g * 720 + rank) * 8 + q)", "? (uint64_t)((g * 720 + rank) * 7 + q)"),
    "h2_random_key_rank_dropped": ("? (uint64_t)((g * 720 + rank) * 8 + q)", "? (uint64_t)((g * 720) * 8 + q)"),
    "h2x_random_key_stride_8": ("+ (uint64_t)rank) * 16u + (uint64_t)q)", "+ (uint64_t)rank) * 8u + (uint64_t)q)"),
    "h2_random_layout_switch_off_by_one": ("seed, s_run <= 6\n", "seed, s_run <= 5\n"),
    "h2_random_layout_by_instance_length": ("seed, s_run <= 6\n", "seed, s <= 6\n"),
    "bounded_newest_closes": ("        or_close_at(active, na, 0);", "        or_close_at(active, na, *na - 1);"),
    "bounded_limit_off_by_one": ("    if (*na >= max_open)\n        or_close_at", "    if (*na > max_open)\n        or_close_at"),
    "bounded_full_bins_stay_open": ("            if (after == cap)              /* completely filled: the bin closes */\n                or_close_at(active, &na, chosen_at);",
                                    "            if (0)\n                or_close_at(active, &na, chosen_at);"),
    "bounded_division_unbounded": ("            if (2 * before < cap && cap <= 2 * after) {\n                or_make_room(active, &na, max_open);",
                                   "            if (2 * before < cap && cap <= 2 * after) {\n                if (na >= max_open) { bins[nb].load = 0; bins[nb].type = bins[chosen].type; ++nb; raw[q] = chosen; continue; }"),
    "presort_ascending": ("        return x->w > y->w ? -1 : 1;", "        return x->w < y->w ? -1 : 1;"),
    "presort_ties_reversed": ("    return x->pos < y->pos ? -1 : (x->pos > y->pos ? 1 : 0);", "    return x->pos > y->pos ? -1 : (x->pos < y->pos ? 1 : 0);"),
    "presort_bins_not_mapped_back": ("                bin_of_item[it[j].pos] = bs[j];", "                bin_of_item[j] = bs[j];"),
    "last_partial_sublist_dropped": ("for (int64_t g = 0; g * s < m; ++g) {", "for (int64_t g = 0; (g + 1) * s <= m; ++g) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    """The mistake planted at every place its anchor occurs."""
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    path = oracle.compile_variant(src.replace(old, new), str(tmp_path / f"mut_{name}.so"))
    bad = failing_pins_isolated(path)
    assert bad, f"planted mistake {name} passed every pin"


# Anchors shared by the unbounded membrane run and the bounded-space run
# (reading G15), which follows it in the source: the same slip planted in the
# bounded run alone must be caught too.
SHARED = sorted(k for k, (old, _) in MUTANTS.items() if oracle.source_text().count(old) == 2)


@pytest.mark.parametrize("name", SHARED)
def test_planted_mistake_in_bounded_run_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    cut = src.index("static int64_t or_membrane_run_bounded(")
    head, tail = src[:cut], src[cut:]
    assert head.count(old) == 1 and tail.count(old) == 1, name
    path = oracle.compile_variant(head + tail.replace(old, new), str(tmp_path / f"mutb_{name}.so"))
    bad = failing_pins_isolated(path)
    assert bad, f"planted mistake {name} (bounded run only) passed every pin"


def test_unmodified_copy_passes(tmp_path):
    path = oracle.compile_variant(oracle.source_text(), str(tmp_path / "same.so"))
    assert failing_pins_isolated(path) == []
