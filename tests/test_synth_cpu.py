"""The synthetic inputs follow their stated recipes (no method arithmetic
here): Hermitian Cholesky vectors and dipoles, the energy partitions, and
the ragged batch of 48 instances."""

import numpy as np

from synth import batched_shapes, make_instance


def test_instance_structure():
    inst = make_instance(6, 14, 40, 30, seed=0)
    nc, nw = 6, 14
    assert np.all(np.abs(inst.B - np.conj(inst.B.transpose(0, 2, 1))) == 0)
    assert np.all(np.abs(inst.dip - np.conj(inst.dip.transpose(0, 2, 1))) == 0)
    core, val, vir = inst.eps[:nc], inst.eps[nc:nc + nw], inst.eps[nc + nw:]
    # metal 2p levels: 2 p1/2 at -29.5 and 4 p3/2 at -28.9 Eh, +-0.01
    assert np.all(np.abs(core[:2] + 29.5) <= 0.01) and np.all(np.abs(core[2:6] + 28.9) <= 0.01)
    # valence energies come in Kramers pairs in (-1.4, -0.3); virtuals in (0.05, 2.5)
    assert np.all(val[0::2] == val[1::2]) and val.min() > -1.4 and val.max() < -0.3
    assert vir.min() > 0.05 and vir.max() < 2.5
    # Cholesky vector scale decays as 0.3 exp(-P / 60)
    r = np.abs(inst.B[20]).std() / np.abs(inst.B[0]).std()
    assert abs(r - np.exp(-20 / 60)) < 0.1


def test_batched_recipe():
    sh = batched_shapes(48)
    assert len(sh) == 48
    for i, s in enumerate(sh):
        assert s["ncore"] == 6 and s["nroots"] == 4 and s["seed"] == 1000 + i
        assert s["nval"] % 2 == 0 and 20 <= s["nval"] <= 80
        assert 100 <= s["nvirt"] <= 400 and s["naux"] == 5 * s["nvirt"]
    assert len({(s["nval"], s["nvirt"]) for s in sh}) > 40  # ragged
