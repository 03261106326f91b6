"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on the same
seeded input and compare everything element by element (all integer: bit-exact)."""
import numpy as np

import oracle


def lambda_bits_from_phi(phi: np.ndarray) -> np.ndarray:
    bits = np.zeros(phi.shape[0], dtype=np.uint64)
    for i in range(phi.shape[1]):
        bits |= (phi[:, i] > 0).astype(np.uint64) << np.uint64(i)
    return bits


def compare_state(h, o, check_phi=True):
    np.testing.assert_array_equal(h.partition(), o.partition())
    np.testing.assert_array_equal(h.block_weights(), o.block_weights())
    assert h.objective() == o.objective()
    if check_phi:
        phi_o = o.phi()
        phi_h = h.phi()
        np.testing.assert_array_equal(phi_h, phi_o)
        np.testing.assert_array_equal(h.lam(), lambda_bits_from_phi(phi_o))
        assert h.objective_from_phi() == o.objective()


def run_both(hg, rounds=None, S=4, seed=0, phi_width=0, part=None, check_phi=True, chunks=None,
             **variant):
    """Refine with both paths; `chunks` splits the rounds into several refine calls;
    `variant` (balance_moves, revert_negative) goes to both."""
    from paper_2010_10272_gb300 import HGP
    rounds = hg.rounds if rounds is None else rounds
    h = HGP.from_hypergraph(hg, part=part, subrounds=S, seed=seed, phi_width=phi_width, **variant)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=seed, part=part, **variant)
    assert h.info()["lmax"] == o.lmax
    compare_state(h, o, check_phi)
    got, want = [], []
    for c in (chunks or [rounds]):
        got.append(h.refine(c)[:, :5])
        want.append(o.refine(c)[0])
    got = np.concatenate(got) if got else np.zeros((0, 5), np.int64)
    want = np.concatenate(want) if want else np.zeros((0, 5), np.int64)
    np.testing.assert_array_equal(got, want)
    compare_state(h, o, check_phi)
    return h, o, got
