"""CPU tests of libppgmres: it loads, exports every symbol the C header
declares, and its host-side steps (harmonic Ritz values, Leja order, root
adding, CSR validation) agree with the oracle.  No GPU needed."""
import os
import re

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import synth
from oracle import poly

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ppg():
    from paper_1911_07065_gb300 import build as B
    B.build()
    import paper_1911_07065_gb300 as p
    return p


def test_library_exports_every_declared_symbol(ppg):
    hdr = open(os.path.join(ROOT, "include", "ppgmres.h")).read()
    declared = set(re.findall(r"\b(ppg_[a-z_0-9]+)\s*\(", hdr))
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(ppg.lib, name), name
    assert declared == set(ppg.EXPORTS)
    assert ppg.lib.ppg_abi_version() == 2
    assert ppg.lib.ppg_strerror(-3).decode() == "H_dd is singular"


def _match(t1, t2):
    C = np.abs(t1[:, None] - t2[None, :])
    r, c = linear_sum_assignment(C)
    return C[r, c], r


def _eig_condition(G):
    import scipy.linalg as sla
    w, vl, vr = sla.eig(G, left=True, right=True)
    s = np.abs(np.sum(vl.conj() * vr, axis=0)) / (np.linalg.norm(vl, axis=0) * np.linalg.norm(vr, axis=0))
    return w, 1.0 / s


@pytest.mark.parametrize("seed,d", [(0, 6), (1, 15), (2, 30), (3, 45)])
def test_harmonic_ritz_matches_oracle_on_same_hbar(ppg, seed, d):
    rng = np.random.default_rng(seed)
    n = 120
    A = rng.standard_normal((n, n)) / np.sqrt(n) + 1.5 * np.eye(n)
    _, H, _ = poly.arnoldi(A, rng.standard_normal(n), d)
    t_lib = ppg.harmonic_ritz(H)
    t_orc = poly.harmonic_ritz(H)
    err, idx = _match(t_lib, t_orc)
    # relative error scaled by the eigenvalue condition number of G
    Hdd = H[:d, :d]
    e = np.zeros(d); e[-1] = 1
    f = np.linalg.solve(Hdd.T, e)
    G = Hdd.copy(); G[:, -1] += H[d, d - 1] ** 2 * f
    w, kappa = _eig_condition(G)
    kap = np.array([kappa[np.argmin(np.abs(w - t))] for t in t_lib[idx]])
    assert np.all(err / np.abs(t_lib[idx]) <= 1e-12 * np.maximum(1.0, kap))
    # exact conjugate structure
    for t in t_lib:
        if t.imag != 0:
            assert np.conj(t) in t_lib


def test_harmonic_ritz_singular_h_is_an_error(ppg):
    H = np.zeros((4, 3))
    H[1, 0] = 1.0
    with pytest.raises(ppg.PPGError) as ei:
        ppg.harmonic_ritz(H)
    assert ei.value.code == -3


def _parse(s):
    return np.array([complex(x.strip()) for x in s.split(",")])


def test_leja_matches_oracle_golden_and_random(ppg):
    for line in open(os.path.join(ROOT, "tests", "golden", "leja_cases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        inp, out = [p.strip() for p in line.split(";")]
        assert np.array_equal(ppg.leja_order(_parse(inp)), _parse(out))
    rng = np.random.default_rng(5)
    for _ in range(30):
        nr, npair = rng.integers(0, 8), rng.integers(0, 6)
        z = rng.uniform(-2, 6, npair) + 1j * rng.uniform(0.05, 3, npair)
        th = np.concatenate([rng.uniform(-1, 8, nr), z, z.conj()]).astype(complex)
        if th.size == 0:
            continue
        rng.shuffle(th)
        assert np.array_equal(ppg.leja_order(th), poly.leja_order(th))


def test_add_roots_matches_oracle_golden_and_random(ppg):
    for line in open(os.path.join(ROOT, "tests", "golden", "root_adding_cases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        inp, out, nadd = [p.strip() for p in line.split(";")]
        r = ppg.add_roots(_parse(inp))
        assert r.n_added == int(nadd)
        assert np.array_equal(r.complex(), _parse(out))
    rng = np.random.default_rng(6)
    for _ in range(20):
        # spectra with outliers so that copies get added
        base = rng.uniform(0.5, 2.0, 30)
        out = rng.uniform(50, 5000, rng.integers(1, 4))
        z = np.array([rng.uniform(1, 2) + 1j * rng.uniform(200, 900)])
        th = poly.leja_order(np.concatenate([base, out, z, z.conj()]))
        ro, nadd, lp = poly.add_roots(th)
        rl = ppg.add_roots(th)
        assert rl.n_added == nadd
        assert np.array_equal(rl.complex(), ro)
        assert np.allclose(rl.pof(), lp, rtol=0, atol=1e-9)


def test_roots_from_hessenberg_example7(ppg):
    """Example 7 through the library's host steps on the oracle's Hbar:
    the two roots added at 30 and 60."""
    A = synth.diag_csr(synth.ex7_diagonal()).to_scipy()
    v0 = synth.gaussian_v0(synth.streams(7)[0], 5000)
    P = poly.build_poly(A, 125, v0)
    r = ppg.roots_from_hessenberg(P.Hbar)
    assert r.n_orig == 125 and r.n_added == 2
    assert np.allclose(np.sort(r.complex()[125:].real), [30, 60], rtol=1e-6)
    err, _ = _match(r.complex(), P.roots)
    assert err.max() / np.abs(P.roots).max() < 1e-10


def test_csr_validation(ppg):
    A = synth.cd2d(7, 0.3)
    assert ppg.csr_validate_host(A.rowptr, A.colind) == 0
    bad = A.colind.copy()
    bad[3] = 49
    assert ppg.csr_validate_host(A.rowptr, bad) == -2
    unsorted = A.colind.copy()
    unsorted[[0, 1]] = unsorted[[1, 0]]
    assert ppg.csr_validate_host(A.rowptr, unsorted) == -2
    rp = A.rowptr.copy()
    rp[5] = rp[6] + 1
    assert ppg.csr_validate_host(rp, A.colind) == -2


def test_header_is_plain_c_and_links(ppg, tmp_path):
    """A C99 program (no C++ anywhere) includes the header, links the
    library and calls host-only entry points: the ABI needs no C++ or torch
    on the caller's side."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include "ppgmres.h"
int main(void) {
    ppg_opts o;
    double re[3] = {1.0, 4.0, 2.0}, im[3] = {0.0, 0.0, 0.0}, ro[3], io[3];
    ppg_default_opts(&o);
    if (ppg_abi_version() != 2 || o.max_cycles <= 0) return 1;
    if (ppg_leja_order(3, re, im, ro, io) != PPG_OK) return 2;
    /* the largest modulus first (modified Leja order) */
    if (ro[0] != 4.0) return 3;
    printf("%s\n", ppg_strerror(PPG_ERR_ARG));
    return 0;
}
''')
    libdir = os.path.dirname(ppg.lib._name)
    exe = tmp_path / "abi"
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lppgmres",
           "-Wl,-rpath," + libdir, "-o", str(exe)]
    subprocess.run(cmd, check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert out.stdout.strip() == ppg.lib.ppg_strerror(-1).decode()
