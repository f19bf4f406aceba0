"""The run-time specialised pricing and sensitivity kernels compile (NVRTC,
sm_103a, no GPU needed) for every test and workload program at its model's
underlying count."""
import pytest

from cases import CASES
import paper_2108_03076_gb300 as pc


@pytest.mark.parametrize("name", sorted(CASES))
def test_specialised_kernel_compiles(name):
    text, tp, spec, _ = CASES[name]
    w, k = pc.pc_assemble(text)
    assert pc.pc_debug_jit_compile(w, k, tp, len(spec.S0)) > 1000


@pytest.mark.parametrize("name", ["european", "lookback", "nested_loops", "double_barrier", "basket_and",
                                  "history_now", "nat_ops"])
def test_specialised_sensitivity_kernel_compiles(name):
    """Loops (loopif frames, fused loop tests), lookbacks, history reads and
    integer arithmetic through the tangent generator's successor jumps."""
    text, tp, spec, _ = CASES[name]
    w, k = pc.pc_assemble(text)
    assert pc.pc_debug_jit_compile(w, k, tp, len(spec.S0), kind=32) > 1000


def test_compile_errors_are_reported():
    w, k = pc.pc_assemble("(model 0 1)")
    with pytest.raises(pc.PcError) as e:
        pc.pc_debug_jit_compile(w, k, [], 5)
    assert e.value.name == "PC_EINVAL"


@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5, 12, 16, 16 + 2, 16 + 4, 16 + 6, 16 + 3, 24, 24 + 2, 24 + 6, 32, 33, 64, 65])
def test_specialised_variants_compile(kind):
    """The per-path, HBM-window, register-window and four-paths-a-lane pricing
    variants, the control-variate kernel in each mode (second-order term,
    pilot sums, per-path outputs; with the window in registers)
    and the sensitivity kernel (sums, per-path) for the worst-of
    autocallable."""
    import workloads as W
    w_ = W.worst_of_autocall()
    w, k = pc.pc_assemble(w_.il_text)
    assert pc.pc_debug_jit_compile(w, k, w_.tparams, 3, kind=kind) > 1000


@pytest.mark.parametrize("kind,d", [(8, 1), (16 + 1, 3), (24 + 1, 3), (16, 4), (34, 1), (31, 1), (14, 1), (66, 1)])
def test_unknown_kinds_are_refused(kind, d):
    w, k = pc.pc_assemble("(model 0 1)")
    with pytest.raises(pc.PcError) as e:
        pc.pc_debug_jit_compile(w, k, [], d, kind=kind)
    assert e.value.name == "PC_EINVAL"


def test_generated_source_is_what_the_compiler_gets():
    """pc_debug_jit_source returns the kernel's CUDA source: one entry point
    per kind, the same text for the same program, another for another."""
    import workloads as W
    w_ = W.worst_of_autocall()
    w, k = pc.pc_assemble(w_.il_text)
    price = pc.pc_debug_jit_source(w, k, w_.tparams, 3, kind=0)
    assert "pc_jit_price" in price and "pc_jit_greeks" not in price
    assert pc.pc_debug_jit_source(w, k, w_.tparams, 3, kind=0) == price
    assert "pc_jit_greeks" in pc.pc_debug_jit_source(w, k, w_.tparams, 3, kind=32)
    assert "pc_jit_cv" in pc.pc_debug_jit_source(w, k, w_.tparams, 3, kind=16)
    w2, k2 = pc.pc_assemble(W.daily_barrier().il_text)
    assert pc.pc_debug_jit_source(w2, k2, W.daily_barrier().tparams, 3, kind=0) != price
    with pytest.raises(pc.PcError) as e:
        pc.pc_debug_jit_source(w, k, w_.tparams, 3, kind=34)
    assert e.value.name == "PC_EINVAL"
