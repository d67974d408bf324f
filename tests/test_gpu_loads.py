"""GPU: the loads of Eq. (3) on axis-aligned box patches from separable 1D
integrals equal the element-by-element quadrature of the same Gauss rule
(different summation order: 1e-12 relative), for every source kind; the
oracle parity of both paths is in test_gpu_parity.py and test_gpu_boundary.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_04340_gb300 import workloads as wl


@pytest.fixture(scope="module")
def ieti():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti as m
    return m


def _patchwise_box():
    rng = np.random.default_rng(11)
    return wl.unit_cube(2, (2, 2, 1), [[2, 3], [3, 2], [2]], sub_of_patch=np.array([0, 1, 0, 1], np.int32),
                        source_kind=wl.SOURCE_PATCHWISE, source_params=rng.standard_normal(3 * 4 * 3), nrhs=3)


def _fourier_box():
    return wl.unit_cube(3, (2, 2, 2), [[2, 3], [3, 2], [2, 2]], source_kind=wl.SOURCE_FOURIER,
                        source_params=wl.fourier_source_params(5, 3, 7, nmodes=9), nrhs=5)


CASES = {
    "sine_cube8_p2n4": lambda: wl.cube8_p2n4(),
    "sine_ragged_p3": lambda: wl.unit_cube(3, (2, 2, 1), [[2, 3], [3, 2], [3]],
                                           sub_of_patch=np.array([0, 1, 0, 2], np.int32), nrhs=2,
                                           source_params=[1.0, -2.0]),
    "fourier_box_p3": _fourier_box,
    "fourier_uneven8": lambda: wl.cube64_uneven8(nrhs=8),
    "trig_paper_cube": lambda: wl.paper_cube(2, 2, nrhs=2, amps=[1.0, -0.5]),
    "patchwise_box": _patchwise_box,
}


def _loads(ieti, prob, element):
    ctx = ieti.ieti_create(prob)
    try:
        if element:
            ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_ELEMENT_LOADS, 1)
        n0 = ieti.ieti_launch_count(ctx)
        ieti.ieti_assemble(ctx)
        n = ieti.ieti_launch_count(ctx) - n0
        nsub = ieti.ieti_query(ctx)["nsub"]
        jr = [ieti.ieti_get_block(ctx, 3, k) for k in range(nsub)]
        jp = [ieti.ieti_get_block(ctx, 4, k) for k in range(nsub)]
        return jr, jp, n
    finally:
        ieti.ieti_destroy(ctx)


@pytest.mark.parametrize("name", list(CASES))
def test_separable_loads_equal_element_quadrature(ieti, name):
    prob = CASES[name]()
    jr_s, jp_s, n_s = _loads(ieti, prob, False)
    jr_e, jp_e, n_e = _loads(ieti, prob, True)
    # the separable path replaces the element kernel by a table, a load and a sum kernel
    assert n_s == n_e + 2
    scale = max(np.abs(b).max() for b in jr_e)
    for a, b in zip(jr_s + jp_s, jr_e + jp_e):
        if b.size:
            assert np.abs(a - b).max() <= 1e-12 * scale


def test_non_integer_wave_numbers_keep_the_element_quadrature(ieti):
    prob = wl.unit_cube(2, (2, 1, 1), 2, source_kind=wl.SOURCE_FOURIER,
                        source_params=[1.0, 0.5, 1.0, 0.0, 0.3, -0.2, 0.1, 0.0, 0.4, 0.2])
    _, _, n_s = _loads(ieti, prob, False)
    _, _, n_e = _loads(ieti, prob, True)
    assert n_s == n_e


@pytest.mark.parametrize("name", ["sine_ragged_p3", "fourier_box_p3", "trig_paper_cube"])
def test_tile_reassembly_equals_first_assembly(ieti, name):
    """After the first factorisation found the nonzero tiles of K_rr, later
    assemblies generate only those (the lower ones, written with their
    mirrors); the blocks equal the full first assembly's to rounding, and the
    separable loads are bit-identical from one assembly to the next."""
    prob = CASES[name]()
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        nsub = ieti.ieti_query(ctx)["nsub"]
        K1 = [ieti.ieti_get_block(ctx, 0, k) for k in range(nsub)]
        j1 = [ieti.ieti_get_block(ctx, 3, k) for k in range(nsub)]
        ieti.ieti_factor(ctx, ieti.IETI_FP64)
        ieti.ieti_assemble(ctx)
        for k in range(nsub):
            K2 = ieti.ieti_get_block(ctx, 0, k)
            assert np.abs(K2 - K1[k]).max() <= 1e-14 * np.abs(K1[k]).max()
            assert np.array_equal(K2, K2.T)
            if name != "trig_paper_cube":   # (its boundary lifting adds with atomics)
                # the patch parts of the loads are summed in a fixed order
                assert np.array_equal(ieti.ieti_get_block(ctx, 3, k), j1[k])
    finally:
        ieti.ieti_destroy(ctx)
