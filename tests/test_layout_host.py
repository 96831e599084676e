"""Host-only layout construction through the C-ABI (``lbm_check_config``;
no GPU): the compact row layout of the workloads passes its built-in
self-check (every population pull resolves to its own stored cell), the
sizes match the inputs, and invalid inputs are rejected with a reason."""
import pytest

from workloads import aorta, configs


@pytest.fixture(scope="module")
def check():
    from paper_2112_05258_gb300 import build as b
    b.build()
    from paper_2112_05258_gb300 import check_config
    return check_config


@pytest.mark.parametrize("filaments", [False, True])
def test_ib_tube_layout(check, filaments):
    inst = configs.ib_tube(filaments=filaments)
    st = check([inst])
    assert st["ib_nodes"] == inst.ib.n
    assert st["filaments"] == (len(inst.ib.filaments) if filaments else 0)
    assert st["fluid_cells"] == inst.n_fluid
    assert 0 < st["band_cells"] <= inst.n_fluid
    # the slab pipeline, when asked for (cuts at planes 4, 8, ..., 20 of the
    # 24-plane tube; every wall node's support passes the slab check);
    # filaments keep the serial step
    assert st["slabs"] == 0
    assert check([inst], ib_slabs=8)["slabs"] == (0 if filaments else 6)


def test_aorta_layout(check):
    inst = aorta.build(0)
    st = check([inst])
    assert st["fluid_cells"] == 4019584 and st["ib_nodes"] == 204566
    assert st["stored_cells"] < st["box_cells"] / 4      # the compact rows skip the solid
    assert st["slabs"] == 0
    assert check([inst], ib_slabs=8)["slabs"] == 8 and check([inst], ib_slabs=16)["slabs"] == 16


def test_batch_sizes_add_up(check):
    insts = [configs.lv_tube(), configs.rigid_tube(16, 16, 24, radius=5.0, period=200), configs.lv_tube_x(31)]
    st = check(insts)
    assert st["band_cells"] == 0 and st["ib_nodes"] == 0 and st["slabs"] == 0
    assert st["fluid_cells"] == sum(i.n_fluid for i in insts)


def test_invalid_configs_are_rejected_with_a_reason(check):
    from paper_2112_05258_gb300 import LBMError
    inst = configs.ib_tube(filaments=True)
    inst.ib.pinned = inst.ib.pinned.copy()
    inst.ib.pinned[inst.ib.filaments[0][0]] = 0
    with pytest.raises(LBMError, match="end nodes must be pinned"):
        check([inst])
    bad = configs.lv_tube()
    bad.tau = 0.5
    with pytest.raises(LBMError):
        check([bad])
