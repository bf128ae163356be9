"""Resource budget of the hot kernels as ptxas reported it when the library
was compiled (no GPU needed): the fine kernels run 256-thread CTAs two to an
SM and the adjoint's reverse kernel 512-thread CTAs one to an SM, so a kernel
that needs more than 128 registers a thread, or spills to local memory, loses
occupancy or bandwidth before it ever runs."""
import re

import pytest


@pytest.fixture(scope="module")
def usage(mmplib):
    from paper_2310_11365_gb300 import build

    u = build.resource_usage()
    if not u:
        pytest.skip("no ptxas reports next to the objects (library built elsewhere)")
    return u


def _select(usage, pattern):
    hits = {k: v for k, v in usage.items() if re.fullmatch(pattern, k)}
    assert hits, pattern
    return hits


@pytest.mark.parametrize("pattern,what", [
    (r"_ZN3mmp6k_fineIfLi0ELb[01]ELi0EEEvNS_8FineArgsE", "mixed fine kernels (shared-memory layout, both noise forms)"),
    (r"_ZN3mmp6k_fineIdLi0ELb[01]ELi0EEEvNS_8FineArgsE", "FP64 fine kernels (shared-memory layout, both noise forms)"),
    (r"_ZN3mmp6k_fineI[fd]Li0ELb0ELi1EEEvNS_8FineArgsE", "plane-rotator fine kernels (mixed and FP64)"),
    (r"_ZN3mmp12k_fine_batchIfLb[01]EEEvNS_9BatchArgsE", "mixed batched fine kernels"),
    (r"_ZN3mmp9k_adjointI[fd]Lb[01]ELi512EEEvNS_11AdjointArgsE", "adjoint reverse kernels (512 threads)"),
])
def test_hot_kernels_fit_two_ctas_per_sm_without_spills(usage, pattern, what):
    for name, rec in _select(usage, pattern).items():
        assert rec["registers"] <= 128, (what, name, rec)
        assert rec.get("spill_stores", 0) == 0 and rec.get("spill_loads", 0) == 0, (what, name, rec)


def test_every_kernel_has_a_report(usage):
    """Every __global__ of the library appears, with its register count."""
    names = " ".join(usage)
    for k in ("k_fine", "k_fine_batch", "k_batch_plan", "k_driver", "k_driver_batch", "k_adjoint",
              "k_init_u0", "k_normals", "k_philox"):
        assert re.search(rf"\d{k}I|\d{k}E", names), k
    assert all(r["registers"] > 0 for r in usage.values())
