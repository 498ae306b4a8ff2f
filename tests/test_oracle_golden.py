"""Oracle vs the hand-worked example in golden/hand_nand_inv.txt (Eq. 1, 2, 6, 7)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from tests.golden.fixtures import load


@pytest.fixture(scope="module")
def case():
    lib, net, v = load("hand_nand_inv.txt")
    return Oracle(net, lib), v


def test_loads_sp_tr_power(case):
    o, v = case
    K = v["K"][0]
    np.testing.assert_allclose(o.cload(), v["cload"], rtol=0, atol=1e-12)
    sp, tr = o.forward(np.array(v["sp_in"]), np.array(v["tr_in"]))
    np.testing.assert_allclose(sp, v["sp"], atol=1e-15)
    np.testing.assert_allclose(tr, v["tr"], atol=1e-15)
    assert o.power(tr, v["vdd"][0], v["fclk"][0]) == pytest.approx(v["power_K"][0] * K, rel=1e-14)


def test_model_gradients(case):
    o, v = case
    K = v["K"][0]
    sp, tr = o.forward(np.array(v["sp_in"]), np.array(v["tr_in"]))
    g = o.backward(np.array(v["sp_in"]), np.array(v["tr_in"]), None, 0, 0, v["vdd"][0], v["fclk"][0])
    np.testing.assert_allclose(g["grad_sp_in"], np.array(v["grad_sp_in_K"]) * K, rtol=1e-13)
    np.testing.assert_allclose(g["grad_tr_in"], np.array(v["grad_tr_in_K"]) * K, rtol=1e-13)
    np.testing.assert_allclose(g["grad_pincap"], np.array(v["grad_pincap_K"]) * K, rtol=1e-13)
    np.testing.assert_allclose(g["grad_cload"], np.array(v["grad_cload_K"]) * K, rtol=1e-13)


@pytest.mark.parametrize("mode,key", [(1, "grad_sp_in_mode1_K"), (2, "grad_sp_in_mode2_K")])
def test_hybrid_gradients(case, mode, key):
    o, v = case
    K = v["K"][0]
    sp, tr = o.forward(np.array(v["sp_in"]), np.array(v["tr_in"]))
    beta = np.array(v["beta"])
    alpha = beta * tr
    assert o.power(alpha, v["vdd"][0], v["fclk"][0]) == pytest.approx(v["power_hybrid_K"][0] * K, rel=1e-14)
    g = o.backward(np.array(v["sp_in"]), np.array(v["tr_in"]), beta, mode, 0, v["vdd"][0], v["fclk"][0])
    np.testing.assert_allclose(g["grad_sp_in"], np.array(v[key]) * K, rtol=1e-13)
    np.testing.assert_allclose(g["grad_tr_in"], np.array(v["grad_tr_in_hybrid_K"]) * K, rtol=1e-13)
    np.testing.assert_allclose(g["grad_pincap"], np.array(v["grad_pincap_hybrid_K"]) * K, rtol=1e-13)
    np.testing.assert_allclose(g["grad_cload"], np.array(v["grad_cload_hybrid_K"]) * K, rtol=1e-13)
