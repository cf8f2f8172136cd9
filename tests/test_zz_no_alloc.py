"""The allocation-free OC entry point against the regular one.

to_oc_update_noalloc serves callers that cannot allocate device memory (it
takes no context and no workspace; its scratch is a static device array of
the library).  Two calls in a row must give the same design update as
to_oc_update, within the OC tolerance of the parity tests (1e-10 absolute on
rho), so leftover scratch contents from the first call cannot leak into the
second.  The test suite's ordering (tests/conftest.py) puts this file last,
so that a run that stops at the first failure has already run every other
test.
"""

import numpy as np
import pytest

from gpu_helpers import Ctx, dev, host
from workloads import small_problem, rand_density

pytestmark = pytest.mark.gpu


def test_noalloc_oc_matches_context_oc_on_two_calls():
    from paper_2205_00385_gb300 import binding as B
    import torch
    p = small_problem("cantilever3d", nelx=48, nely=24, nelz=24, mg_levels=3, volfrac=0.12)
    nel = p.nel
    rng = np.random.default_rng(385)
    with Ctx(p, precision="fp64") as c:
        dvf = dev(np.zeros(nel))
        B.to_filter(c.ctx, B.TO_FILTER_SENS, dev(np.ones(nel)), dvf)
        rho0 = rand_density(nel, 31, 0.05, 0.4)
        rho_ctx, rho_na = dev(rho0), dev(rho0)
        for call in range(2):
            dc = -rng.uniform(0.01, 5.0, nel)
            dcf = dev(np.zeros(nel))
            B.to_filter(c.ctx, B.TO_FILTER_SENS, dev(dc), dcf)
            ch_ctx, ch_na = dev(np.zeros(1)), dev(np.zeros(1))
            B.to_oc_update(c.ctx, p.volfrac, 0.2, dcf, dvf, rho_ctx, ch_ctx)
            B.to_oc_update_noalloc(nel, p.volfrac, 0.2, dcf, dvf, rho_na, ch_na,
                                   torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            a, b = host(rho_ctx), host(rho_na)
            assert np.max(np.abs(a - b)) <= 1e-10, call
            assert abs(host(ch_ctx)[0] - host(ch_na)[0]) <= 1e-10, call
            # the update did move the design and kept the volume
            assert host(ch_na)[0] > 0.0
            assert abs(host(dvf) @ b - p.volfrac * nel) <= 1e-8 * p.volfrac * nel


def test_noalloc_oc_rejects_sizes_beyond_capacity():
    from paper_2205_00385_gb300 import binding as B
    import torch
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(B.TopoError) as e:
        B.to_oc_update_noalloc((1 << 21) + 1, 0.3, 0.2, x, x, x, None,
                               torch.cuda.current_stream().cuda_stream)
    assert e.value.status == B.TO_E_INVALID
    assert "capacity" in B.to_last_error(None)
