"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/pepic.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pepic.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"PE_API\s+[\w\s\*]+?\b(pe_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1610_01071_gb300 import _build

    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    names = declared_symbols()
    for required in ("pe_create", "pe_burst", "pe_restrict", "pe_project", "pe_lift", "pe_step",
                     "pe_deposit", "pe_field", "pe_push", "pe_sample", "pe_coarsen", "pe_ls_project",
                     "pe_refine", "pe_quiet_start", "pe_sort"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(lib):
    from paper_1610_01071_gb300 import _binding

    assert sorted(_binding.SIGNATURES) == declared_symbols()


def test_library_exports_nothing_else(lib):
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_1610_01071_gb300", "libpepic.so")],
                         capture_output=True, text=True).stdout
    exported = sorted({l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("pe_")})
    assert exported == declared_symbols()


def test_layout_is_host_only_and_validates(lib):
    from paper_1610_01071_gb300 import _binding as b

    cfg = b.make_config(4096, 256, 20, 1 << 24, 2048.0, 0.1, 20.0)
    lay = b.layout(cfg)
    assert lay.total_bytes >= 2 * 16 * (1 << 24)
    offs = list(lay.offset)
    assert offs == sorted(offs) and all(o % 256 == 0 for o in offs)
    bad = b.make_config(4000, 256, 20, 1 << 24, 2048.0, 0.1, 20.0)
    with pytest.raises(b.PepicError):
        b.layout(bad)
    assert lib.pe_strerror is not None


def test_kinetic_electron_layout_and_checks(lib):
    from paper_1610_01071_gb300 import _binding as b

    base = (64, 16, 4, 64 * 16, 32.0, 0.005, 0.1)
    for bad in (dict(boundary="absorbing"),   # kinetic electrons: periodic grids only
                dict(poisson="linearized"),   # the lifting's Boltzmann relation is exponential
                dict(qm_e=5.0), dict(v_th_e=-1.0), dict(reset_every=-1)):
        with pytest.raises(b.PepicError):
            b.layout(b.make_config(*base, electrons="kinetic", **bad))
    lay = b.layout(b.make_config(*base, electrons="kinetic"))
    bank = 4 * ((4 * 64 * 16 + 255) // 256) * 256
    assert lay.bytes[b.BUF["electrons_a"]] == bank and lay.bytes[b.BUF["electrons_b"]] == bank
    assert lay.bytes[b.BUF["rho_e"]] == 8 * 3 * 64  # electron deposit + the ions' moments [2][ncell]
    lay0 = b.layout(b.make_config(*base))
    assert lay0.bytes[b.BUF["electrons_a"]] == 0 and lay0.bytes[b.BUF["rho_e"]] == 0
    assert lay.total_bytes >= lay0.total_bytes + 2 * bank


def test_a_c_program_links_and_calls_the_host_entry_points(lib, tmp_path):
    # the boundary is plain C: a C99 program includes the header, links libpepic and calls the
    # host-only entry points (no GPU needed)
    import shutil
    import subprocess

    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "pepic.h"
int main(void) {
    pe_config c;
    memset(&c, 0, sizeof c);
    c.ncell = 4096; c.n_coarse = 256; c.wavelet = PE_WAVELET_HAAR; c.K = 20;
    c.nparticles = (int64_t)1 << 24; c.L = 2048.0; c.dt = 0.1; c.dT = 20.0; c.qm = 1.0; c.v_th = 1.0;
    c.comoving = 1; c.poisson = PE_POISSON_BOLTZMANN; c.newton_tol = 1e-10; c.newton_maxit = 50;
    pe_layout lay;
    int rc = pe_layout_for(&c, &lay);
    c.ncell = 4000;
    int bad = pe_layout_for(&c, &lay);
    printf("%s|%d|%d|%s|%zu\n", pe_version(), rc, bad, pe_strerror(PE_EINVAL), lay.total_bytes > 0 ? (size_t)1 : (size_t)0);
    return rc == PE_OK && bad == PE_EINVAL ? 0 : 1;
}
""")
    libdir = os.path.join(ROOT, "paper_1610_01071_gb300")
    exe = tmp_path / "abi"
    cuda_lib = "/usr/local/cuda/lib64"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe), "-L", libdir, "-lpepic", "-Wl,-rpath," + libdir, "-Wl,-rpath," + cuda_lib],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, run.stdout + run.stderr
    version, rc, bad, msg, _ = run.stdout.strip().split("|")
    assert version.startswith("pepic") and rc == "0" and bad == "1" and msg


def test_layout_of_the_phase_space_wavelet_form(lib):
    # n_v fine velocity cells in the sample rows, n_v_coarse coefficients in the coarse state,
    # and the fine-node sampling tables; configurations outside the form are refused
    from paper_1610_01071_gb300 import _binding as b

    def cfg(**kw):
        a = dict(coarse="phase_space", n_v=256, v_max=8.0, n_v_coarse=64, wavelet="coif4")
        a.update(kw)
        return b.make_config(4096, 256, 20, 1 << 24, 2048.0, 0.1, 8.0, **a)

    lay = b.layout(cfg())
    assert lay.bytes[b.BUF["samples_fx"]] == 8 * 256 * 256 * 22  # [K+2][n_coarse][n_vf]
    assert lay.bytes[b.BUF["coarse"]] == 8 * 256 * 64  # [n_coarse][n_vc]
    haar = b.layout(cfg(n_v_coarse=0, wavelet="haar"))
    assert lay.bytes[b.BUF["phase"]] >= haar.bytes[b.BUF["phase"]] + 4 * 4096 * (3 * 256 + 1)
    for bad in (dict(n_v_coarse=128, n_v=64), dict(n_v=200), dict(ps_filter=1), dict(boundary="absorbing"),
                dict(electrons="kinetic"), dict(n_v_coarse=1), dict(n_v_coarse=48)):
        with pytest.raises(RuntimeError):
            b.layout(cfg(**bad))
    with pytest.raises(RuntimeError):  # the wavelet form belongs to the phase-space variable
        b.layout(b.make_config(4096, 256, 20, 1 << 24, 2048.0, 0.1, 8.0, n_v_coarse=16))


def test_layout_of_the_pressure_variable(lib):
    # three nodal moment rows per sample, [3][n_coarse] coarse state, (n, u, T) profiles; the
    # kind is refused on bounded grids, with kinetic electrons and above 4096 cells
    from paper_1610_01071_gb300 import _binding as b

    def cfg(**kw):
        a = dict(ncell=4096, n_coarse=256, K=20, nparticles=1 << 24, L=2048.0, dt=0.1, dT=20.0,
                 coarse="moments_pressure")
        a.update(kw)
        return b.make_config(**a)

    lay = b.layout(cfg())
    assert lay.bytes[b.BUF["samples_fx"]] == 8 * 3 * 4096 * 22  # [K+2][3][ncell]
    assert lay.bytes[b.BUF["coarse"]] == 8 * 3 * 256
    assert lay.bytes[b.BUF["profile"]] == 4 * 3 * 4096
    for bad in (dict(boundary="absorbing"), dict(electrons="kinetic"),
                dict(ncell=8192, nparticles=1 << 25, n_coarse=512, L=4096.0)):
        with pytest.raises(RuntimeError):
            b.layout(cfg(**bad))
    s_e = ctypes.c_int32()
    assert lib.pe_second_moment_shift(ctypes.c_int64(1 << 24), 4096, ctypes.c_double(0.0), ctypes.c_double(0.0),
                                      ctypes.byref(s_e)) == 0
    # the largest |w V~^2| = (8 ncell / N) 32^2 = 2 maps to 2^22
    assert s_e.value == 21
