"""The oracle's pins have teeth: each plausible mistake planted in a copy of the
oracle's C source (an off-by-one, a dropped term, a wrong sign or index, a
swapped operand) makes at least one pin fail.  The mutants are compiled on the
CPU into a temporary directory; the committed oracle is untouched."""
import contextlib
import os
import subprocess

import pytest

import oracle
import test_oracle_pairs as pair_pins
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "aln_oracle.c")

MUTANTS = {
    "lf_lower_bound_row": ("occ(t, c, (int64_t)k - 1) + 1", "occ(t, c, (int64_t)k) + 1"),
    "insertion_window": ("i >= e && i <= m - 1 - e", "i >= e && i <= m - e"),
    "deletion_window": ("i >= e1 && i <= m - e1", "i >= e1 - 1 && i <= m - e1"),
    "no_gap_extension": ("if (last == OP_I) {", "if (0) {"),
    "d_prune_off_by_one": ("c->budget - diffs < c->D[i]", "c->budget - diffs <= c->D[i]"),
    "n_matches_a": ("if (c->q[i] == b)", "if ((c->q[i] & 3) == b)"),
    "seed_ignores_deletion": ("dfs(c, i, kk[b], ll[b], n_mm, n_gapo + 1, n_gape, n_ins, n_del + 1, seed2, OP_D)",
                              "dfs(c, i, kk[b], ll[b], n_mm, n_gapo + 1, n_gape, n_ins, n_del + 1, seed, OP_D)"),
    "witness_gapo_order": ("return a->n_gapo < b->n_gapo", "return a->n_gapo > b->n_gapo"),
    "c1_stratum": ("all[i].n_diff == d_best + 1", "all[i].n_diff == d_best + 2"),
    "reverse_not_complemented": ("(strand ? (uint8_t)(3 - b) : b)", "b"),
    "dscan_overcounts": ("            cnt++;\n", "            cnt += 2;\n"),
    "bucket_pads_with_t": ("key = 4 * key + (i + j < n ? text[i + j] : 0);", "key = 4 * key + (i + j < n ? text[i + j] : 3);"),
    "bucket_key_drops_symbol": ("for (int j = 0; j < bk; j++) key", "for (int j = 1; j < bk; j++) key"),
    "mix64_shift": ("z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBULL;"),
    "pair_insert_without_len": ("return (int64_t)v->pos + (int64_t)v->len - (int64_t)f->pos;",
                                "return (int64_t)v->pos - (int64_t)f->pos;"),
    "pair_window_3iqr": ("int64_t lo = (int64_t)st->q1 - 2 * iqr, hi = (int64_t)st->q3 + 2 * iqr;",
                         "int64_t lo = (int64_t)st->q1 - 3 * iqr, hi = (int64_t)st->q3 + 3 * iqr;"),
    "pair_median_index": ("st->q2 = ins[u / 2];", "st->q2 = ins[(u + 1) / 2];"),
    "pair_tie_far_from_median": ("else if (e != eb) better = e < eb;", "else if (e != eb) better = e > eb;"),
    "pair_same_strand_is_fr": ("*fr = a->strand != b->strand;", "*fr = 1;"),
    "pair_reverse_pos_no_len": ("out[k].pos = h[j].strand ? ix->t[0].sa[row] : n - ix->t[1].sa[row] - h[j].aligned_len;",
                                "out[k].pos = h[j].strand ? ix->t[0].sa[row] : n - ix->t[1].sa[row];"),
    "score_gapo_weight": ("return p->sc_mm * h->n_mm + p->sc_gapo * h->n_gapo + p->sc_gape * h->n_gape;",
                          "return p->sc_mm * h->n_mm + p->sc_gape * h->n_gapo + p->sc_gape * h->n_gape;"),
    "score_second_stratum": ("if (sc > s1 && (s2 < 0 || sc < s2)) s2 = sc;", "if (sc >= s1 && (s2 < 0 || sc < s2)) s2 = sc;"),
    "score_many_best_inclusive": ("int many = p->max_best > 0 && c0 > (uint64_t)p->max_best;",
                                  "int many = p->max_best > 0 && c0 >= (uint64_t)p->max_best;"),
    "dollar_largest": ("return li < lj ? -1 : (li > lj ? 1 : 0);", "return li > lj ? -1 : (li < lj ? 1 : 0);"),
    "best1_no_second_stratum": ("int keep_max = (p->strata == 1) ? z : (d_best + 1 <= z ? d_best + 1 : z);",
                                "int keep_max = (p->strata == 1) ? z : d_best;"),
    "forward_position_offset": ("n - ix->t[1].sa[row] - h[i].aligned_len", "n - ix->t[1].sa[row] - h[i].aligned_len + 1"),
    "order_strand_before_diffs": ("if (x->n_diff != y->n_diff) return x->n_diff < y->n_diff ? -1 : 1;\n    if (x->strand != y->strand)",
                                  "if (x->strand != y->strand) return x->strand < y->strand ? -1 : 1;\n    if (x->n_diff != y->n_diff)"),
    "mismatch_seed_free": ("else if (seed_ok)\n            dfs(c, i + 1, kk[b], ll[b], n_mm + 1, n_gapo, n_gape, n_ins, n_del, seed2, OP_M);",
                           "else\n            dfs(c, i + 1, kk[b], ll[b], n_mm + 1, n_gapo, n_gape, n_ins, n_del, seed, OP_M);"),
}


def _pin_calls():
    c = pins.CASES
    return [
        pins.test_hand_example,
        pins.test_mix64_matches_published_splitmix64,
        lambda: pins.test_sa_bwt_against_naive_sort(300, 4, 2, 3),
        lambda: pins.test_exact_interval_is_naive_scan(21),
        pins.test_z0_is_exact_matching,
        lambda: pins.test_mismatch_only_is_hamming_scan(2),
        lambda: pins.test_against_brute_force(*c[1], "FULL"),
        lambda: pins.test_against_brute_force(*c[3], "BEST1"),
        lambda: pins.test_against_brute_force(*c[5], "FULL"),
        pins.test_positions_match_brute_force,
        pins.test_d_array_properties_and_safety,
        pins.test_best1_is_full_filtered,
        pins.test_edge_reads,
        pins.test_homopolymer_gap_witness,
        lambda: pins.test_every_position_every_edit(0),
        lambda: pins.test_every_position_every_edit(2),
        lambda: pins.test_against_brute_force(*c[2], "FULL"),
        lambda: pins.test_every_pair_of_edits_in_seed(1),
        lambda: pins.test_score_mode_against_brute_force(0),
        lambda: pins.test_score_mode_against_brute_force(2),
        pair_pins.test_pairing_hand_example,
        pair_pins.test_pairing_recovers_the_generated_fragments,
    ]


@contextlib.contextmanager
def _oracle_from(path):
    saved_lib, saved_build = oracle._lib, oracle.build
    oracle._lib = None
    oracle.build = lambda force=False: path
    try:
        yield
    finally:
        oracle._lib, oracle.build = saved_lib, saved_build


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mut = src.replace(old, new, 1)
    c_path = tmp_path / "mut.c"
    so_path = tmp_path / "libmut.so"
    c_path.write_text(mut)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-shared",
                           "-fPIC", "-pthread", "-o", str(so_path), str(c_path)])
    caught = []
    with _oracle_from(str(so_path)):
        for call in _pin_calls():
            try:
                call()
            except (AssertionError, ValueError, IndexError):
                caught.append(call)
                break
    assert caught, f"mutant {name} passed every pin"
