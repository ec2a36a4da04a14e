"""The algorithmic operation counts behind the roofline numerator.  The oracle
evaluates its own formulas once with a counting number type (orc_flop_counts) and
reports, by category, the additions, multiplications, divisions, exponentials,
logarithms and powers of one right-hand-side evaluation, one analytic Jacobian, one
LU factorisation and one solve.  The LU and solve counts equal the closed forms of
Doolittle elimination; the bench's structural model (bench.flop_model), which the
roofline uses, is checked against them: equal for LU and solve, and never above the
oracle's plain formulas for the rates and the Jacobian (which evaluate a logarithm
and a power per reaction and a dense Jacobian), so the roofline numerator does not
overstate the work."""
import numpy as np
import pytest

import bench
import mechgen

E = bench.FLOPS_PER_TRANSCENDENTAL


def arith(d):
    return d["add"] + d["mul"] + d["div"]


def transc(d):
    return d["exp"] + d["log"] + 2 * d["pow"]      # a power is a logarithm and an exponential


@pytest.mark.parametrize("which", ["small", "medium", "large"])
def test_counts_and_the_structural_model(orc, which):
    spec = {"small": mechgen.MECH_SMALL, "medium": mechgen.MECH_MEDIUM, "large": mechgen.MECH_LARGE}[which]
    mech = mechgen.make_mechanism({"small": 1000, "medium": 3000, "large": 5000}[which], **spec)
    m = orc.Mech(mech)
    rng = np.random.default_rng(2)
    y = np.concatenate([rng.dirichlet(np.ones(mech.n_species)), [1500.0]])
    c = m.flop_counts(y, 101325.0, 2e-9)
    n = mech.n
    # Doolittle LU with partial pivoting: sum_k (n-k-1)^2 multiply-adds and sum_k (n-k-1) divisions;
    # forward and backward substitution: n(n-1) multiply-adds and n divisions
    mad = (n - 1) * n * (2 * n - 1) // 6
    assert c["lu"] == dict(add=mad, mul=mad, div=n * (n - 1) // 2, exp=0, log=0, pow=0)
    assert c["solve"] == dict(add=n * (n - 1), mul=n * (n - 1), div=n, exp=0, log=0, pow=0)
    fm = bench.flop_model(mech)
    assert fm["lu"] == arith(c["lu"])
    assert fm["solve"] == arith(c["solve"])
    # rates: the model's transcendentals (one exponential per reaction for k_f, one per
    # species factor for K_c, seven per falloff reaction, ln T) and arithmetic stay below
    # the oracle's formulas
    R, ntroe = mech.n_reactions, int((mech.rtype == 2).sum())
    model_transc = 2 * R + 7 * ntroe + 1
    assert model_transc <= transc(c["rhs"])
    assert fm["rates"] - E * model_transc <= arith(c["rhs"])
    # the Jacobian with its rate evaluation
    jac_model = fm["rates"] + fm["jac_fp64"] + fm["jac_asm"]
    assert jac_model <= arith(c["jac"]) + E * transc(c["jac"])


def test_per_substep_count_of_the_box_workload(orc):
    """The figure quoted in the design notes: FP64 flops per cell-step of the box
    mechanism under the minimal policy (I Newton iterations, J Jacobians per substep),
    from the model and from the oracle's counts."""
    w = mechgen.workload("box32")
    m = orc.Mech(w.mech)
    c = m.flop_counts(w.y0[1000], w.p[1000], 5e-9 * 0.4358665215)
    fm = bench.flop_model(w.mech)
    I, J = 7.11, 0.167
    model = I * (fm["rates"] + fm["solve"] + fm["vec"]) + J * (fm["rates"] + fm["jac_fp64"] + fm["jac_asm"] + fm["lu"])
    flops = {k: arith(v) + E * transc(v) for k, v in c.items()}
    oracle_count = I * (flops["rhs"] + flops["solve"] + fm["vec"]) + J * (flops["jac"] + flops["lu"])
    print(f"box mechanism, {I} Newton and {J} Jacobians per substep: model {model:.4g}, oracle formulas "
          f"{oracle_count:.4g} FP64 flops per cell-step")
    assert 1.3e5 < model < 1.6e5
    assert model < oracle_count
