"""Helpers for the GPU parity tests: build a library context for a workload
and move arrays between numpy and the device.  Calls go through the C ABI
(``paper_2205_00385_gb300.binding``)."""

from __future__ import annotations

import numpy as np


def torch():
    import torch as t
    return t


def dev(a, dtype=None):
    t = torch()
    x = t.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        x = x.to(dtype)
    return x.to("cuda")


def host(x):
    return x.detach().cpu().numpy()


class Ctx:
    """A libtopo context for a workloads.Problem, plus its workspace."""

    def __init__(self, prob, precision=None, levels=None):
        from paper_2205_00385_gb300 import binding as B
        t = torch()
        self.B = B
        self.prob = prob
        prec = precision or prob.precision
        self.desc = B.make_desc(prob.dim, (prob.nelx, prob.nely, prob.nelz), prob.E0, prob.Emin,
                                prob.nu, prob.penal, prob.rmin,
                                levels if levels is not None else prob.mg_levels,
                                B.TO_MIXED if prec == "mixed" else B.TO_FP64, prob.n_parm,
                                prob.n_carm)
        nbytes = B.to_workspace_bytes(self.desc)
        raw = t.empty(nbytes + 256, dtype=t.uint8, device="cuda")
        off = (-raw.data_ptr()) % 256
        self.raw = raw
        self.ws = raw[off:off + nbytes]
        self.fixed = dev(prob.fixed.astype(np.uint8))
        self.f = dev(prob.f.astype(np.float64))
        self.stream = t.cuda.current_stream()
        self.ctx = B.to_mesh_init(self.desc, self.fixed, self.f, self.ws, self.stream.cuda_stream)

    def set_density(self, rho_phys):
        self.B.to_set_density(self.ctx, dev(np.asarray(rho_phys, np.float64)))

    def close(self):
        if self.ctx is not None:
            self.B.to_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
