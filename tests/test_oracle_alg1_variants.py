"""Pins of the closest-match and sorted-search forms of Alg. 1 (section 3.1,
the variants after the listing)."""
import numpy as np
import pytest

import problems as P
from oracle import psr_oracle as O


def patches(pr):
    return O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())


CASES = [("diff3d", lambda: P.diffusion3d_q2(4, sigma=0.5, corr_len=3.0, seed=1), 0.2),
         ("diff3d_loose", lambda: P.diffusion3d_q2(4, sigma=0.5, corr_len=3.0, seed=1), 0.6),
         ("stokes", lambda: P.stokes2d_q2q1(8, 1.05), 0.05),
         ("poisson", lambda: P.poisson2d_q2(8), 1e-12)]


@pytest.mark.parametrize("name,make,tol", CASES)
def test_closest_match_keeps_the_entries_and_takes_the_nearest_passing_one(name, make, tol):
    """Brute force: the representatives are Alg. 1's; phi(i) of a non-rep
    patch is the argmin of d over the entries created before it among those
    with d < tol (lowest j on ties)."""
    A = patches(make())
    a = O.alg1(A, tol)
    c = O.alg1_closest_match(A, tol)
    assert np.array_equal(a["reps"], c["reps"]) and c["near_ties"] == []
    reps = c["reps"]
    Binv = c["Binv"]
    for i in range(A.shape[0]):
        if i in set(reps.tolist()):
            assert reps[c["phi"][i]] == i
            continue
        live = np.flatnonzero(reps < i)
        d = np.array([O.criterion(A[i][None], A[reps[j]][None], Binv[j][None])[0] for j in live])
        ok = live[d < tol]
        assert ok.size and c["phi"][i] == ok[np.argmin(d[d < tol])]


def test_closest_and_first_match_differ_on_scaled_copies():
    """Copies s A of one patch: d(s_i A, s_j A) = |1 - s_i / s_j|.  With
    s = 1, 1.5, 1.3 and tol 0.4 the third patch passes both entries (0.3 and
    0.133): first match takes entry 0, closest match entry 1."""
    A0 = patches(P.poisson2d_q2(4))[5]
    A = np.stack([A0, 1.5 * A0, 1.3 * A0])
    a = O.alg1(A, 0.4)
    c = O.alg1_closest_match(A, 0.4)
    assert a["reps"].tolist() == c["reps"].tolist() == [0, 1]
    assert a["phi"].tolist() == [0, 1, 0] and c["phi"].tolist() == [0, 1, 1]


@pytest.mark.parametrize("name,make,tol", CASES)
def test_sorted_search_equals_alg1_with_fewer_tests(name, make, tol):
    A = patches(make())
    a = O.alg1(A, tol)
    s = O.alg1_sorted(A, tol)
    assert np.array_equal(a["phi"], s["phi"]) and np.array_equal(a["reps"], s["reps"])
    assert s["evals"] <= a["evals"]


def test_norm_window_is_necessary():
    """Every pair with d < tol lies in the window
    ||A||/(1+tol) < ||B|| < ||A||/(1-tol), checked on all pairs of a
    random-coefficient problem at several tolerances."""
    A = patches(P.diffusion3d_q2(3, sigma=1.0, corr_len=2.0, seed=5))
    nrm = np.array([np.linalg.svd(a, compute_uv=False)[0] for a in A])
    Binv, _ = O.lu_inverse(A)
    for j in range(A.shape[0]):
        d = O.criterion(A, np.repeat(A[j][None], A.shape[0], axis=0), np.repeat(Binv[j][None], A.shape[0], axis=0))
        for tol in (0.05, 0.3, 0.8):
            inside = (nrm / (1 + tol) < nrm[j] * (1 + 1e-12)) & (nrm[j] * (1 - 1e-12) < nrm / (1 - tol))
            assert np.all(inside[d < tol])
