"""Planted mistakes: each plausible slip in the oracle's arithmetic (a dropped
term, a wrong shift amount or direction, a transposed operand or index, a
wrong operator, a missing step) is planted in a copy of oracle/ci_oracle.c,
compiled on the CPU, and the pins named beside it must fail against that copy
(the unmodified oracle passes the same pins in the rest of the suite).  This
shows that the pins tell the oracle from a near miss of it, not only that the
oracle agrees with itself."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ci_oracle.c")

# (id, text in ci_oracle.c, planted text, pins: test node ids under tests/)
MUTANTS = [
    # Eq. (Oplus)
    ("ci_step_or_for_xor", "return x ^ strategy;", "return x | strategy;",
     ["test_oracle_ci.py::test_table1_worked_example"]),
    # Algorithm 2 (XORshift)
    ("xorshift32_shift_amount", "z = z ^ (z << 13);", "z = z ^ (z << 12);",
     ["test_oracle_xorlike.py::test_xorshift32_full_period_gf2"]),
    ("xorshift32_shift_direction", "z = z ^ (z >> 17);", "z = z ^ (z << 17);",
     ["test_oracle_xorlike.py::test_xorshift32_full_period_gf2"]),
    # xor128 (Sec. 6.2) and xor64 (Sec. 7)
    ("xor128_shift_amount", "uint32_t tmp = a ^ (a << 11);", "uint32_t tmp = a ^ (a << 12);",
     ["test_oracle_xorlike.py::test_xor128_full_period_gf2"]),
    ("xor128_dropped_term", "s[3] = s[3] ^ (s[3] >> 19) ^ (tmp ^ (tmp >> 8));", "s[3] = s[3] ^ (tmp ^ (tmp >> 8));",
     ["test_oracle_xorlike.py::test_xor128_full_period_gf2"]),
    ("xor64_shift_amount", "x = x ^ (x >> 7);", "x = x ^ (x >> 8);",
     ["test_oracle_xorlike.py::test_xor64_full_period_gf2"]),
    # Algorithm 4: the mixing
    ("mix_dropped_partner", "tnew[l] = xl[l] ^ tprev[part1[l]] ^ tprev[part2[l]];",
     "tnew[l] = xl[l] ^ tprev[part1[l]];",
     ["test_oracle_mixing.py::test_hand_worked_c2_synchronous", "test_oracle_mixing.py::test_hand_worked_c4"]),
    ("mix_asynchronous_reading", "tnew[l] = xl[l] ^ tprev[part1[l]] ^ tprev[part2[l]];",
     "tnew[l] = tprev[l] = xl[l] ^ tprev[part1[l]] ^ tprev[part2[l]];",
     ["test_oracle_mixing.py::test_hand_worked_c2_synchronous", "test_oracle_mixing.py::test_hand_worked_c4"]),
    ("ci_update_with_own_word", "x[l] = orc_ci_step(x[l], tnew[l]);", "x[l] = orc_ci_step(x[l], xl[l]);",
     ["test_oracle_mixing.py::test_hand_worked_c2_synchronous"]),
    ("mix_second_array_read_from_first", "p2[l] = base + c2[offset];", "p2[l] = base + c1[offset];",
     ["test_oracle_mixing.py::test_partner_indexing_impulse_xor"]),
    ("mix_group_base_dropped", "p1[l] = base + c1[offset];", "p1[l] = c1[offset];",
     ["test_oracle_mixing.py::test_partner_indexing_impulse_xor"]),
    # BBS and Algorithm 5
    ("bbs_square_wrong_modulus", "return (uint64_t)(sq % (unsigned __int128)M);",
     "return (uint64_t)(sq % (unsigned __int128)(M - 1));",
     ["test_oracle_bbs.py::test_bbs_step_large_moduli"]),
    ("bbs_chunk_one_bit_short", "t |= (uint32_t)(orc_bbs_next(s) & mask);",
     "t |= (uint32_t)(orc_bbs_next(s) & (mask >> 1));",
     ["test_oracle_bbs.py::test_assembly_w4_matches_algorithm5_text", "test_oracle_bbs.py::test_assembly_w5"]),
    ("bbs_shift_draw_one_bit", "uint32_t shift = (uint32_t)(orc_bbs_next(s) & 3u);",
     "uint32_t shift = (uint32_t)(orc_bbs_next(s) & 1u);",
     ["test_oracle_bbs.py::test_assembly_w4_matches_algorithm5_text", "test_oracle_bbs.py::test_assembly_w5"]),
    ("bbs_array_shift_entry", "static const uint32_t array_shift[4] = {0u, 1u, 3u, 7u};",
     "static const uint32_t array_shift[4] = {0u, 1u, 3u, 3u};",
     ["test_oracle_bbs.py::test_assembly_w4_matches_algorithm5_text", "test_oracle_bbs.py::test_assembly_w5"]),
    ("bbs_second_array_precedence", "c2 = comb + (size_t)(8 + lanes[l].sel2) * C;",
     "c2 = comb + (size_t)((8 + lanes[l].sel2) & 7u) * C;",
     ["test_oracle_mixing.py::test_partner_indexing_impulse_bbs"]),
    ("bbs_bits_per_step_rounded_up", "while ((lg >> w) > 1)", "while ((lg >> w) > 0)",
     ["test_oracle_bbs.py::test_secure_bit_count"]),
    ("bbs_prime_not_3_mod_4", "p = (uint32_t)((1ULL << 30) + (d >> 34)) | 3u;",
     "p = (uint32_t)((1ULL << 30) + (d >> 34)) | 1u;",
     ["test_oracle_bbs.py::test_seeded_lanes_have_blum_primes"]),
    ("bbs_second_selector_bits", "L->sel2 = (uint32_t)((v >> 3) & 7);", "L->sel2 = (uint32_t)((v >> 4) & 7);",
     ["test_oracle_bbs.py::test_seeded_lanes_have_blum_primes"]),
    ("bbs16_prime_range", "p = (uint32_t)(128 + d % 128) | 3u;", "p = (uint32_t)(128 + d % 256) | 3u;",
     ["test_oracle_bbs16.py::test_seeded_generators"]),
    ("trial_division_misses_squares", "for (uint64_t d = 3; d * d <= n; d += 2)",
     "for (uint64_t d = 3; d * d < n; d += 2)",
     ["test_oracle_bbs.py::test_trial_division_matches_library"]),
    # Algorithm 5 as printed
    ("bbs16_second_array_precedence", "c2 = comb + (size_t)(8 + (lanes[l].y16[1] & 7u)) * C;",
     "c2 = comb + (size_t)((8 + lanes[l].y16[1]) & 7u) * C;",
     ["test_oracle_bbs16.py::test_recurrence_with_arrays_chosen_per_call"]),
    ("bbs16_rotation_missing", "orc_bbs16_rotate(&lanes[l]);", ";",
     ["test_oracle_bbs16.py::test_squaring_counts_and_rotation_after_a_call"]),
    ("bbs16_shift_from_wrong_generator", "shift = orc_bbs16_next(L, 2) & 3u;", "shift = orc_bbs16_next(L, 3) & 3u;",
     ["test_oracle_bbs16.py::test_hand_worked_word_fixes_generator_order"]),
    ("bbs16_nibble_three_bits", "t |= orc_bbs16_next(L, k) & 15u;", "t |= orc_bbs16_next(L, k) & 7u;",
     ["test_oracle_bbs16.py::test_hand_worked_word_fixes_generator_order"]),
    # the quarter-circle consumer and the seeding counter layout
    ("qc_fixed_point_shift", "uint64_t a = held[l] >> 8, b = xs[l] >> 8;",
     "uint64_t a = held[l] >> 7, b = xs[l] >> 8;",
     ["test_oracle_seeding_stats.py::test_qc_counts_equal_real_number_test"]),
    ("qc_threshold", "if (a * a + b * b < (1ULL << 48))", "if (a * a + b * b < (1ULL << 47))",
     ["test_oracle_seeding_stats.py::test_qc_counts_equal_real_number_test"]),
    ("qc_pairs_shifted_by_one", "if ((i & 1) == 0) {", "if ((i & 1) == 1) {",
     ["test_oracle_seeding_stats.py::test_qc_counts_equal_real_number_test"]),
    ("lane_counter_overlap", "return orc_draw(seed, (lane << 32) + k);", "return orc_draw(seed, (lane << 31) + k);",
     ["test_oracle_seeding_stats.py::test_lane_counter_ranges"]),
    # chaotic Blum-Goldwasser (Sec. 9.2)
    ("bg_keystream_without_s0", "uint32_t k = S0;", "uint32_t k = 0;",
     ["test_oracle_bg.py::test_keystream_is_prefix_xor_of_bbs_bits"]),
    ("bg_chunk_one_bit_short", "k ^= (uint32_t)(x & mask);", "k ^= (uint32_t)(x & (mask >> 1));",
     ["test_oracle_bg.py::test_keystream_is_prefix_xor_of_bbs_bits"]),
    ("bg_decryption_keystream_without_s0", "uint64_t x = orc_bg_recover_x0(p, q, y, L);\n    uint32_t k = S0;",
     "uint64_t x = orc_bg_recover_x0(p, q, y, L);\n    uint32_t k = 0;",
     ["test_oracle_bg.py::test_round_trip_and_paper_sized_key"]),
    ("bg_crt_inverse_transposed", "orc_invmod(q % p, p)", "orc_invmod(p % q, q)",
     ["test_oracle_bg.py::test_crt_recovers_x0"]),
    ("bg_root_exponent_power_off_by_one", "orc_powmod((p + 1) / 4, L, p - 1)", "orc_powmod((p + 1) / 4, L + 1, p - 1)",
     ["test_oracle_bg.py::test_crt_recovers_x0"]),
    # Listing 1 / Algorithm 3
    ("listing1_dropped_high_halves", "return x ^ (uint32_t)T ^ (uint32_t)(T >> 32);", "return x ^ (uint32_t)T;",
     ["test_oracle_naive.py::test_listing1_combination_hand_worked"]),
    ("listing1_dropped_generator", "const uint64_t T = t1 ^ t2 ^ t3;", "const uint64_t T = t1 ^ t2;",
     ["test_oracle_naive.py::test_listing1_combination_hand_worked"]),
    ("naive_xor128_shift_amount", "T t = s[0] ^ (s[0] << 11);", "T t = s[0] ^ (s[0] << 10);",
     ["test_oracle_naive.py::test_xor128_instances_share_the_pinned_recurrence"]),
    ("naive_xorshift_shift_amount", "T t = s[0] ^ (s[0] >> 7);", "T t = s[0] ^ (s[0] >> 6);",
     ["test_oracle_naive.py::test_xorshift160_full_period"]),
    ("naive_xorwow_shift_amount", "s[4] = (s[4] ^ (s[4] << 4)) ^ (t ^ (t << 1));",
     "s[4] = (s[4] ^ (s[4] << 5)) ^ (t ^ (t << 1));",
     ["test_oracle_naive.py::test_xorwow_linear_part_full_period"]),
    # published first outputs (splitmix64, xor128, xor64) and the output
    # functions of Listing 1's five-word xorshift and xorwow
    ("splitmix64_multiplier", "0xBF58476D1CE4E5B9ULL", "0xBF58476D1CE4E5B5ULL",
     ["test_oracle_published.py::test_splitmix64_published_outputs"]),
    ("splitmix64_shift", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBULL;",
     ["test_oracle_published.py::test_splitmix64_published_outputs"]),
    ("splitmix64_gamma", "#define ORC_GAMMA 0x9E3779B97F4A7C15ULL", "#define ORC_GAMMA 0x9E3779B97F4A7C17ULL",
     ["test_oracle_published.py::test_splitmix64_published_outputs"]),
    ("splitmix64_counter_from_zero", "return orc_mix64(seed + (index + 1) * ORC_GAMMA);",
     "return orc_mix64(seed + index * ORC_GAMMA);",
     ["test_oracle_published.py::test_splitmix64_published_outputs"]),
    ("xor128_triple_reversed",
     "uint32_t tmp = a ^ (a << 11);\n    s[0] = s[1];\n    s[1] = s[2];\n    s[2] = s[3];\n"
     "    s[3] = s[3] ^ (s[3] >> 19) ^ (tmp ^ (tmp >> 8));",
     "uint32_t tmp = a ^ (a << 19);\n    s[0] = s[1];\n    s[1] = s[2];\n    s[2] = s[3];\n"
     "    s[3] = s[3] ^ (s[3] >> 11) ^ (tmp ^ (tmp >> 8));",
     ["test_oracle_published.py::test_xor128_published_outputs"]),
    ("xor128_right_shifts_swapped", "s[3] = s[3] ^ (s[3] >> 19) ^ (tmp ^ (tmp >> 8));",
     "s[3] = s[3] ^ (s[3] >> 8) ^ (tmp ^ (tmp >> 19));",
     ["test_oracle_published.py::test_xor128_published_outputs"]),
    ("xor64_triple_reversed", "x = x ^ (x << 13);\n    x = x ^ (x >> 7);\n    x = x ^ (x << 17);",
     "x = x ^ (x << 17);\n    x = x ^ (x >> 7);\n    x = x ^ (x << 13);",
     ["test_oracle_published.py::test_xor64_published_outputs"]),
    ("naive_xs160_output_multiplier_word", "return (T)((T)(s[1] + s[1] + 1u) * s[4]);",
     "return (T)((T)(s[2] + s[2] + 1u) * s[4]);",
     ["test_oracle_published.py::test_xorshift160_32_output_is_odd_multiple_of_newest_word"]),
    ("naive_xs160_output_even_multiplier", "return (T)((T)(s[1] + s[1] + 1u) * s[4]);",
     "return (T)((T)(s[1] + s[1]) * s[4]);",
     ["test_oracle_published.py::test_xorshift160_32_output_is_odd_multiple_of_newest_word"]),
    ("naive_xs160_output_old_word", "return (T)((T)(s[1] + s[1] + 1u) * s[4]);",
     "return (T)((T)(s[1] + s[1] + 1u) * s[3]);",
     ["test_oracle_published.py::test_xorshift160_32_output_is_odd_multiple_of_newest_word"]),
    ("naive_xorwow_output_xor", "return (T)(*d + s[4]);", "return (T)(*d ^ s[4]);",
     ["test_oracle_published.py::test_xorwow32_output_is_weyl_plus_newest_word"]),
    ("naive_xorwow_output_old_word", "return (T)(*d + s[4]);", "return (T)(*d + s[3]);",
     ["test_oracle_published.py::test_xorwow32_output_is_weyl_plus_newest_word"]),
    ("naive_xorwow_output_before_weyl_step", "return (T)(*d + s[4]);", "return (T)(*d - 362437u + s[4]);",
     ["test_oracle_published.py::test_xorwow32_output_is_weyl_plus_newest_word"]),
]


def _cc():
    return os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")


@pytest.mark.skipif(_cc() is None, reason="no host C compiler")
@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pins(name, old, new, pins, tmp_path):
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) >= 1, "the text to mutate is not in the oracle: %r" % old
    c_file, so_file = tmp_path / "planted.c", tmp_path / "libplanted.so"
    c_file.write_text(src.replace(old, new, 1))
    subprocess.check_call([_cc(), "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so_file), str(c_file)])
    env = dict(os.environ, CI_ORACLE_LIB=str(so_file))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x"] + [os.path.join(ROOT, "tests", p) for p in pins],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    summary = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else r.stderr[-500:]
    assert r.returncode == 1 and "failed" in summary, (
        "planted mistake %s was not caught by %s: %s" % (name, pins, summary))
