"""Host-side rules that need no GPU: the T_control block-size rule (Sec. 4.4)."""
import pytest


@pytest.fixture(scope="module")
def C():
    from paper_1607_05707_gb300 import _build, irgl

    _build.build_irgl()
    irgl.lib()
    return irgl


def test_control_cta_intersection(C):
    ALL = 0b1111
    assert C.irgl_control_cta([ALL, ALL]) == 1024                  # several candidates: the highest
    assert C.irgl_control_cta([ALL, ALL], preferred=256) == 256    # unless the preferred one is allowed
    assert C.irgl_control_cta([0b0011, 0b0110]) == 256             # {128,256} & {256,512}
    assert C.irgl_control_cta([0b0011, 0b0110], preferred=1024) == 256
    assert C.irgl_control_cta([0b0100]) == 512                     # FixedBlock kernel
    assert C.irgl_control_cta([]) == 1024                          # no constraint
    with pytest.raises(C.IrglError) as ei:
        C.irgl_control_cta([0b0001, 0b0010])                        # empty: no outlining
    assert ei.value.status == C.IRGL_ERR_UNSUPPORTED
