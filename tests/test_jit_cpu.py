"""The run-time specialised pricing kernel compiles (NVRTC, sm_103a, no GPU
needed) for every test and workload program at its model's underlying
count."""
import pytest

from cases import CASES
import paper_2108_03076_gb300 as pc


@pytest.mark.parametrize("name", sorted(CASES))
def test_specialised_kernel_compiles(name):
    text, tp, spec, _ = CASES[name]
    w, k = pc.pc_assemble(text)
    assert pc.pc_debug_jit_compile(w, k, tp, len(spec.S0)) > 1000


def test_compile_errors_are_reported():
    w, k = pc.pc_assemble("(model 0 1)")
    with pytest.raises(pc.PcError) as e:
        pc.pc_debug_jit_compile(w, k, [], 5)
    assert e.value.name == "PC_EINVAL"
