"""The algorithmic bytes per node update that bench.py's roofline uses follow from the buffer
layout the library reports (no GPU work): populations read and written once, the phase entry
written once and read once."""
import ctypes as C

import pytest

import bench


@pytest.fixture(scope="module")
def abi():
    import paper_1804_08923_gb300.build as b
    b.build()
    from paper_1804_08923_gb300 import _abi
    return _abi


def per_node(abi, storage, n=(64, 32, 48)):
    g = abi.make_grid(*n, abi.BC_PERIODIC, abi.BC_PERIODIC)
    p = abi.make_params(dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.1, nu_b=0.1, storage=storage))
    sizes = (C.c_size_t * abi.MAX_BUFFERS)()
    cnt = C.c_int32()
    assert abi.library().lb_buffer_sizes(C.byref(g), C.byref(p), sizes, C.byref(cnt)) == 0
    nodes = n[0] * n[1] * n[2]
    # buffers 0 and 1: the two population buffers; buffer 2: the phase entries (one per
    # population buffer for the FP16 encodings); buffer 5: the collision moments
    pop = sizes[0] / nodes
    phase = sizes[2] / nodes / (1 if storage == abi.STORE_FP32 else 2)
    mom = sizes[5] / nodes
    return pop, phase, mom


def test_step_bytes_match_the_layout(abi):
    pop, phase, mom = per_node(abi, abi.STORE_FP32)
    assert (pop, phase, mom) == pytest.approx((216, 8, 48), abs=0.01)
    assert bench.BYTES_STEP == 2 * pop + 2 * phase
    assert bench.BYTES_KERNEL["collide_kernel"] == pop + phase + mom
    assert bench.BYTES_KERNEL["moment_kernel"] == pop + phase + mom
    for st, step, kern in ((abi.STORE_FP16, bench.BYTES_STEP_FP16, bench.BYTES_KERNEL_FP16),
                           (abi.STORE_FP16_FIT, bench.BYTES_STEP_FIT, bench.BYTES_KERNEL_FIT)):
        pop, phase, mom = per_node(abi, st)
        assert (pop, phase, mom) == pytest.approx((112, 16, 48), abs=0.01)
        assert step == 2 * pop + 2 * phase
        assert kern["collide_kernel"] == pop + phase + mom
        assert kern["moment_kernel"] == pop + 2 * phase + mom


def test_profile_hash_covers_the_kernels_own_sources(tmp_path):
    """A committed ncu summary stays valid while the sources its kernel is built from are
    unchanged: the headers and the kernel's translation unit, not the others."""
    import shutil
    src = tmp_path / "csrc"
    shutil.copytree(bench.os.path.join(bench.ROOT, "paper_1804_08923_gb300", "csrc"), src)
    before = {k: bench.kernel_source_sha(k, str(src)) for k in ("collide_kernel", "step_kernel", "adj_collide_kernel")}
    assert before["collide_kernel"] == bench.kernel_source_sha("moment_kernel_fp16", str(src))
    assert len(set(before.values())) == 3
    with open(src / "lbcm_adjoint.cu", "a") as f:
        f.write("\n")
    after = {k: bench.kernel_source_sha(k, str(src)) for k in before}
    assert after["collide_kernel"] == before["collide_kernel"] and after["step_kernel"] == before["step_kernel"]
    assert after["adj_collide_kernel"] != before["adj_collide_kernel"]
    with open(src / "lbcm_device.cuh", "a") as f:
        f.write("\n")
    assert all(bench.kernel_source_sha(k, str(src)) != after[k] for k in after)
