"""The autotuner times every applicable kernel configuration and keeps the
fastest; the configuration it picks gives oracle-exact amplitudes."""
import math

import numpy as np
import pytest

import oracle
import pcv_inputs as pin

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autotuner_picks_a_correct_fastest_configuration(tmp_path):
    from paper_2204_00602_gb300 import autotune
    tuner = autotune.Autotuner(path=str(tmp_path / "table.json"), reps=2)
    for m, n, cnt in [(12, 6, 2000), (24, 11, 300)]:
        U = pin.haar_unitary(m, 500 + n)
        t = pin.single_photon_input(m, n)
        outs = pin.random_bunched_outputs(m, n, cnt, 600 + n)
        Ud, od = torch.from_numpy(U).cuda(), torch.from_numpy(outs).cuda()
        algo, param, times = tuner.tune(Ud, t, od)
        assert len(times) == len(autotune.candidates(m, n, cnt)) >= 3
        assert times[(algo, param)] == min(times.values())
        amp, _ = tuner.amplitudes_tuned(Ud, t, od)
        torch.cuda.synchronize()
        a_ref = oracle.amplitudes(U, t, outs)
        floor = 1 / math.sqrt(math.comb(m + n - 1, n))
        assert np.max(np.abs(amp.cpu().numpy() - a_ref) / np.maximum(np.abs(a_ref), floor)) <= 1e-10
    tuner.save()
    again = autotune.Autotuner(path=str(tmp_path / "table.json"))
    assert again.lookup(12, 6, 2000) == tuner.lookup(12, 6, 2000)
