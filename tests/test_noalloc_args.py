"""Argument checks of the no-allocation CG entry point's binding, made on the
host before the library is called (CPU only): every wrong dtype, shape,
layout, device or overlap is refused with ValueError."""
import pytest
import torch

from paper_2210_06874_gb300 import hmc

L, Nt = 2, 4
V = 2 * L * L
CPU = torch.device("cpu")


def good():
    return dict(E=torch.zeros((V, V), dtype=torch.float64),
                phi=torch.zeros((Nt, V), dtype=torch.float64),
                chi=torch.zeros((Nt, V), dtype=torch.complex128),
                x=torch.zeros((Nt, V), dtype=torch.complex128))


def check(**kw):
    a = good()
    a.update(kw)
    hmc.check_noalloc_args(a["E"], L, Nt, a["phi"], a["chi"], a["x"], CPU)


def test_good_arguments_pass():
    check()


@pytest.mark.parametrize("name,bad", [
    ("E", torch.zeros((V, V), dtype=torch.float32)),
    ("E", torch.zeros((V, V - 1), dtype=torch.float64)),
    ("E", torch.zeros((V, 2 * V), dtype=torch.float64)[:, ::2]),
    ("phi", torch.zeros((Nt, V), dtype=torch.complex128)),
    ("phi", torch.zeros((Nt + 1, V), dtype=torch.float64)),
    ("chi", torch.zeros((Nt, V), dtype=torch.complex64)),
    ("chi", torch.zeros((V, Nt), dtype=torch.complex128).t()),
    ("x", torch.zeros((Nt, V), dtype=torch.float64)),
    ("x", torch.zeros((Nt * V,), dtype=torch.complex128)),
    ("x", torch.zeros((Nt, V), dtype=torch.complex128, device="meta")),
    ("E", [[0.0]]),
])
def test_bad_argument_refused(name, bad):
    with pytest.raises(ValueError):
        check(**{name: bad})


def test_overlap_refused():
    buf = torch.zeros((2 * Nt, V), dtype=torch.complex128)
    with pytest.raises(ValueError):
        check(chi=buf[:Nt], x=buf[Nt // 2:Nt // 2 + Nt])
    with pytest.raises(ValueError):
        a = good()
        check(chi=a["chi"], x=a["chi"])


def test_bad_sizes_refused():
    a = good()
    with pytest.raises(ValueError):
        hmc.check_noalloc_args(a["E"], 0, Nt, a["phi"], a["chi"], a["x"], CPU)
    with pytest.raises(ValueError):
        hmc.check_noalloc_args(a["E"], L, 2.5, a["phi"], a["chi"], a["x"], CPU)
