"""Comparison of a CUDA result with the oracle, used by the GPU parity tests.

Two bounds, both asserted:
* relative L2, ||got - ref||_2 / ||ref||_2 <= tol (the stated tolerance of the
  form under test);
* per element, max |got - ref| <= K_ELEM * tol * max |ref|, so that a wrong
  value confined to a few cells (one leaf, one face) cannot hide in the
  2-norm of a large mesh.  For errors spread like rounding, the largest
  deviation is a few times the RMS one, and max |ref| >= RMS |ref|, so
  K_ELEM = 10 leaves room for the tail of the rounding distribution only.
"""
import numpy as np

K_ELEM = 10.0


def rel_l2(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def max_elem(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def assert_close(got, ref, tol, what="", k_elem=K_ELEM):
    e2, em = rel_l2(got, ref), max_elem(got, ref)
    print(f"{what}: rel L2 {e2:.3e} (tol {tol:.1e}), max |d| / max |ref| {em:.3e} (bound {k_elem * tol:.1e})")
    assert e2 <= tol, (what, "rel L2", e2, tol)
    assert em <= k_elem * tol, (what, "per element", em, k_elem * tol)


def corner_and_interior_leaves(L, extra, seed):
    """The 8 corner leaves of a level-L tree ((z, y, x)) plus `extra` interior
    leaves drawn with the given seed."""
    n = 2 ** L
    c = [[z, y, x] for z in (0, n - 1) for y in (0, n - 1) for x in (0, n - 1)]
    rng = np.random.default_rng(seed)
    c += rng.integers(1, n - 1, (extra, 3)).tolist()
    return np.array(c)


def leaf_values(phi, acc, leaves, S):
    """(k, 4, S^3) values of the given leaves from full-mesh outputs."""
    g = np.concatenate([np.asarray(phi)[None], np.asarray(acc)])
    return np.stack([g[:, a * S:(a + 1) * S, b * S:(b + 1) * S, c * S:(c + 1) * S].reshape(4, -1)
                     for a, b, c in leaves])
