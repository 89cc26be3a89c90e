"""The FP64 NumPy network oracle against central finite differences (CPU)."""
import numpy as np
import pytest

import mpnn_oracle as MO
from paper_2308_15020_gb300 import gen


def _tiny():
    return gen.concat([gen.random_ksat(12, 30, 3, 1), gen.random_xor(12, 3, 3, 5, 1, signs=True),
                       gen.random_atleast(12, 2, 4, 6, 1)])


@pytest.mark.parametrize("layers", [1, 2])
def test_gradient_matches_central_differences(layers):
    inst = _tiny()
    _, total = MO.layout(layers)
    rng = np.random.default_rng(layers)
    p = rng.normal(0, 0.3, total)
    t = np.where(rng.random(inst.n) < 0.5, -1.0, 1.0)
    loss, g, x0 = MO.loss_and_grad(p, inst, t, layers, bf16_weights=False, bf16_inputs=False)
    assert np.all(np.abs(x0) <= 1)
    for i in rng.choice(total, size=40, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (MO.loss_and_grad(pp, inst, t, layers, False, False)[0] -
              MO.loss_and_grad(pm, inst, t, layers, False, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.001953125, -3.14159, 65504.0])
    r = MO.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0  # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even
    assert r[2] == 1.0
    assert abs(r[3] + 3.140625) < 1e-12


def test_bf16_inputs_change_only_rounding():
    """Rounding the dense-product inputs to BF16 moves the loss, the proposal
    and every gradient block by rounding-sized amounts only (a dropped or
    misplaced term would move a block by its own size); the rounding is
    idempotent."""
    inst = _tiny()
    layers = 2
    lay, total = MO.layout(layers)
    rng = np.random.default_rng(7)
    p = rng.normal(0, 0.1, total)  # small weights: few ReLU masks flip under the rounding
    t = np.where(rng.random(inst.n) < 0.5, -1.0, 1.0)
    l0, g0, x0 = MO.loss_and_grad(p, inst, t, layers, True, False)
    l1, g1, x1 = MO.loss_and_grad(p, inst, t, layers, True, True)
    assert l0 != l1 and abs(l1 - l0) <= 1e-4 * abs(l0)
    assert np.max(np.abs(x1 - x0)) <= 1e-3
    for name, (o, shape) in lay.items():
        a, b = g0[o:o + int(np.prod(shape))], g1[o:o + int(np.prod(shape))]
        scale = np.max(np.abs(a)) + 1e-12
        assert np.max(np.abs(a - b)) <= 0.05 * scale, name
    v = np.array([0.123456, -7.654321, 1e-3])
    assert np.array_equal(MO.bf16(MO.bf16(v)), MO.bf16(v))
