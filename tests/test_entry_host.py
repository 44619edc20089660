"""Host-side logic of the learned-entry workflow (no GPU)."""
import numpy as np

from paper_2507_17094_gb300.entry import choose_tau


def test_choose_tau_is_the_fallback_quantile():
    rng = np.random.default_rng(3)
    pmax = rng.uniform(0.0, 1.0, 10_000)
    tau = choose_tau(pmax, 0.05)
    assert tau in pmax
    # exactly the chosen fraction sits below the threshold (values are distinct)
    assert (pmax < tau).sum() == int(np.floor(0.05 * (len(pmax) - 1)))
    assert choose_tau(pmax, 0.0) == 0.0
    assert choose_tau(np.array([]), 0.05) == 0.0
    assert choose_tau(pmax, 1.0) == pmax.max()
