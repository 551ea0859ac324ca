"""The oracle's pins catch plausible mistakes.  Each case compiles the oracle
with one deliberate mistake planted (compile-time switch GQ_ORC_MUT in
oracle/gq_oracle.c, never set in normal builds), runs the pin meant to catch
it against that build in a separate process, and requires it to fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gq_oracle.c")

# planted mistake -> the pin (test file, -k expression) that must fail
CASES = {
    1: ("the M2L a_0 term with the sign as printed (Sec. 3.1, eq. m2l)", "test_oracle_math.py", "test_m2l_sign_of_log_term"),
    2: ("M2M binomial index shifted: C(m, k-1) for C(m-1, k-1)", "test_oracle_math.py", "test_m2m_exact"),
    3: ("P2M for S without the 1/k", "test_oracle_math.py", "test_p2m_matches_direct_far_field"),
    4: ("L2L shifting by -y", "test_oracle_math.py", "test_l2l_is_exact_recentering"),
    5: ("D local coefficients d / w^m instead of d / w^(m+1)", "test_oracle_math.py",
        "test_p2l_local_is_taylor_of_potential"),
    6: ("touching boxes treated as not adjacent", "test_oracle_lists.py", "test_touching_same_level_leaves_in_list1"),
    7: ("on-surface value the sum of the two sides, not their mean", "test_oracle_math.py",
        "test_unit_circle_closed_forms"),
    8: ("association threshold slack instead of slack^2", "test_oracle_lists.py", "test_association_bruteforce"),
    9: ("M2L binomial C(m+k-1, k) for C(m+k-1, k-1) in the a_k terms (eq. m2l)", "test_oracle_math.py",
        "test_lemma1_m2qbxl_bound"),
    10: ("List 3 far boxes with few sources not demoted to List 3 close (Remark 1)", "test_oracle_lists.py",
         "test_o2_lists_equal_bruteforce"),
    11: ("S' without the factor m of the derivative of (t - c)^m", "test_oracle_neumann.py",
         "test_unit_circle_neumann_closed_form"),
    12: ("D multipole with w^k for w^(k-1) (eq. multipole)", "test_oracle_math.py",
         "test_p2m_matches_direct_far_field"),
    13: ("TCR(a) < b tested without the factor (1 + t_f) on TCR(a) (Def. 8)", "test_oracle_lists.py",
         "test_list_bounds_and_separation"),
    14: ("a < TCR(b) tested without the factor (1 + t_f) on TCR(b) (Def. 5)", "test_oracle_lists.py",
         "test_list_bounds_and_separation"),
    15: ("centre level from the box itself instead of its TCR (Sec. 4.3)", "test_oracle_lists.py",
         "test_tree_invariants"),
    16: ("centre level from the centre point, the disk radius left out (Sec. 4.3)", "test_oracle_lists.py",
         "test_tree_invariants"),
    17: ("expansion radius from half the panel length, radius_factor x h_k with h_k = arc/2 (Sec. 2.2.2)",
         "test_oracle_math.py", "test_unit_circle_centres"),
    18: ("centre 2i on the exterior side, 2i+1 on the interior (Sec. 2.2.2 ordering)", "test_oracle_math.py",
         "test_unit_circle_centres"),
    19: ("level restriction blind to boxes touching only at a corner (Sec. 4.6 remark)",
         "test_oracle_level_restrict.py", "test_balanced_tree_has_no_violation"),
    20: ("disk-shaped TCR: separation without clamping the overlap along an axis to zero",
         "test_oracle_tcr_disk.py", "test_disk_separation_is_the_geometric_relation"),
    21: ("disk-shaped TCR: centre level from the l-inf distance, as for the square TCR",
         "test_oracle_tcr_disk.py", "test_centre_disks_fit_their_disk_tcr"),
}


@pytest.mark.parametrize("k", sorted(CASES))
def test_planted_mistake_is_caught(k, tmp_path):
    what, test_file, expr = CASES[k]
    lib = str(tmp_path / f"libgq_oracle_mut{k}.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           f"-DGQ_ORC_MUT={k}", "-o", lib, SRC, "-lm"])
    env = dict(os.environ, GQ_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", test_file), "-q", "-x", "-k", expr,
                        "-m", "not gpu", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 1 and " failed" in r.stdout, (what, r.stdout[-2000:])
