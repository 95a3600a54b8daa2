"""The synthetic inputs follow their stated recipes (no method arithmetic
here): Hermitian Cholesky vectors and dipoles, the energy partitions, the
stated and the physical Cholesky scales, and the ragged batch of 48
instances."""

import numpy as np

from synth import batched_shapes, make_instance, physical_scale


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


def test_cholesky_scales():
    # the stated scale: B^0 entries are N(0,1) (+ i N(0,1)) times 0.3
    a = make_instance(2, 4, 10, 3, seed=1)
    off = a.B[0][np.triu_indices(a.B.shape[1], 1)]
    assert 0.2 < np.std(off.real) / 0.3 < 5.0
    # the physical scale 0.34 (nval nvirt^2)^(-1/4): the same draws, scaled
    sc = physical_scale(4, 10)
    assert abs(sc - 0.34 * (4 * 100) ** -0.25) < 1e-15
    assert abs(physical_scale(0, 10) - 0.34 * 100 ** -0.25) < 1e-15
    b = make_instance(2, 4, 10, 3, seed=1, scale=sc)
    assert np.array_equal(a.eps, b.eps)
    assert np.allclose(b.B, a.B * (sc / 0.3), rtol=1e-15, atol=0)
