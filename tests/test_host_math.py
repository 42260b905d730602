"""CPU checks of the library's host-side numerics (csrc/host_math.cpp), compiled on its
own with the host C++ compiler: the level ladder against the paper's level counts
(Sec. 4.3.3), the Chebyshev schedule against the closed-form error polynomial of the
semi-iteration (Sec. 2.3), the dense coarsest-level operator against a Kronecker
construction of the periodic 7-point stencil, and the minimum-norm inverse of the
coarsest solve against numpy's pseudo-inverse and its defining identities, and the
convergence monitor of the solve loops on residual sequences built to end each way."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2607_10983_gb300", "csrc")


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("host") / "host_math_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-Werror", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "host", "host_math_check.cpp"),
                    os.path.join(CSRC, "host_math.cpp"), "-o", exe], check=True)

    def call(*lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return [np.array(line.split(), dtype=np.float64) for line in out.stdout.splitlines()]
    return call


def test_level_ladder(run):
    golden = {}
    with open(os.path.join(ROOT, "tests", "golden", "levels.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n, L = map(int, line.split())
                golden[n] = L
    outs = run(*[f"levels {n} {n} {n} 0" for n in golden])
    for (n, L), v in zip(golden.items(), outs):
        dims = v.reshape(-1, 3).astype(int)
        assert len(dims) == L
        assert (dims == (n >> np.arange(L))[:, None]).all()
    (r96,), (rect,), (lim,) = run("levels 96 96 96 0"), run("levels 64 32 16 0"), run("levels 512 512 512 3")
    assert r96.reshape(-1, 3)[:, 0].astype(int).tolist() == [96, 48, 24, 12, 6]
    assert rect.reshape(-1, 3).astype(int).tolist() == [[64, 32, 16], [32, 16, 8], [16, 8, 4]]
    assert lim.reshape(-1, 3)[:, 0].astype(int).tolist() == [512, 256, 128]


@pytest.mark.parametrize("degree", [1, 2, 3, 4, 6])
def test_chebyshev_schedule_gives_the_chebyshev_error_polynomial(run, degree):
    # the semi-iteration x <- x + d, d <- c1 d + c2 (b - mu x) on a mode of D^-1 A with
    # eigenvalue mu leaves the residual factor T_v((theta - mu)/delta) / T_v(theta/delta)
    alpha = 8.0
    (v,) = run(f"cheb {degree} {alpha}")
    c1, c2 = v[:degree], v[degree:]
    a, b = 2.0 / alpha, 2.0
    theta, delta = (a + b) / 2, (b - a) / 2
    mu = np.linspace(0.0, 2.5, 41)
    x = np.zeros_like(mu)
    d = np.zeros_like(mu)
    for k in range(degree):
        d = c1[k] * d + c2[k] * (1.0 - mu * x)
        x = x + d
    Tv = np.polynomial.chebyshev.Chebyshev.basis(degree)
    ref = Tv((theta - mu) / delta) / Tv(theta / delta)
    np.testing.assert_allclose(1.0 - mu * x, ref, rtol=0, atol=1e-13)


def test_dense_flat_is_the_periodic_7_point_operator(run):
    nx, ny, nz, h = 4, 6, 8, 2.0
    (v,) = run(f"flat {nx} {ny} {nz} {h}")

    def d1(n):
        return np.roll(np.eye(n), 1, axis=1) + np.roll(np.eye(n), -1, axis=1) - 2 * np.eye(n)
    ref = (np.kron(np.kron(np.eye(nz), np.eye(ny)), d1(nx)) + np.kron(np.kron(np.eye(nz), d1(ny)), np.eye(nx))
           + np.kron(np.kron(d1(nz), np.eye(ny)), np.eye(nx))) / h ** 2
    np.testing.assert_array_equal(v.reshape(ref.shape), ref)


def _pinv_call(run, L, w):
    n = len(w)
    (v,) = run("pinv %d %s %s" % (n, " ".join("%.17g" % x for x in w), " ".join("%.17g" % x for x in L.ravel())))
    return int(v[0]), v[1:].reshape(n, n) if v[0] else None


def test_dense_pinv_of_the_flat_coarsest_operator_is_the_pseudo_inverse(run):
    (v,) = run("flat 4 4 4 8")
    L = v.reshape(64, 64)
    ok, G = _pinv_call(run, L, np.ones(64))
    assert ok
    P = np.linalg.pinv(L)
    assert np.abs(G - P).max() < 1e-12 * np.abs(P).max()


def test_dense_pinv_identities_on_a_nonsymmetric_singular_operator(run):
    # L with null space span(1) and left null space span(w): L G r = r - w (w.r)/(w.w), 1^T G r = 0
    rng = np.random.default_rng(7)
    n = 27
    w = rng.uniform(0.5, 1.5, n)
    one = np.ones(n)
    Pw = np.eye(n) - np.outer(w, w) / (w @ w)
    P1 = np.eye(n) - np.outer(one, one) / n
    L = Pw @ (rng.standard_normal((n, n)) + n * np.eye(n)) @ P1
    ok, G = _pinv_call(run, L, w)
    assert ok
    r = rng.standard_normal(n)
    np.testing.assert_allclose(L @ (G @ r), Pw @ r, rtol=0, atol=1e-12 * np.abs(r).max())
    assert abs(one @ (G @ r)) < 1e-12 * np.abs(G @ r).max()
    # a bordered system that is singular is reported, not inverted
    ok0, _ = _pinv_call(run, np.zeros((4, 4)), np.ones(4))
    assert ok0 == 0


def _status_codes():
    codes = {}
    with open(os.path.join(ROOT, "include", "gbmg.h")) as fh:
        for line in fh:
            part = line.split("/*")[0].strip().rstrip(",")
            if part.startswith("GBMG_") and "=" in part:
                name, val = (x.strip() for x in part.split("="))
                codes[name] = int(val)
    return codes


@pytest.mark.parametrize("case", ["converged", "at_start", "budget", "nonfinite", "diverged", "slow_growth",
                                  "long"])
def test_convergence_monitor(run, case):
    S = _status_codes()
    geo = [0.1 ** k for k in range(8)]                         # 1 ... 1e-7
    tol, maxv, seq, want_status, want_cycles = {
        "converged": (2e-6, 100, geo, "GBMG_OK", 6),
        "at_start": (1e-6, 100, [1e-7, 1.0], "GBMG_OK", 0),
        "budget": (1e-12, 3, [2.0 ** -k for k in range(10)], "GBMG_ERR_NOT_CONVERGED", 3),
        "nonfinite": (1e-6, 100, [1.0, 0.5, float("nan"), 0.1], "GBMG_ERR_NONFINITE", 2),
        # tenfold growth over two cycles stops the solve at once; slower growth does not
        "diverged": (1e-6, 100, [1.0, 0.5, 0.9, 5.01, 0.01], "GBMG_ERR_DIVERGED", 3),
        "slow_growth": (1e-6, 100, [1.0, 0.5, 9.9, 4.9, 1e-7], "GBMG_OK", 4),
        "long": (1e-30, 80, [0.9 ** k for k in range(100)], "GBMG_ERR_NOT_CONVERGED", 80),
    }[case]
    line = "monitor %r %d %d %s" % (tol, maxv, len(seq), " ".join(repr(float(x)) for x in seq))
    (v,) = run(line)
    status, cycles = int(v[0]), int(v[1])
    assert status == S[want_status] and cycles == want_cycles
    assert v[2] == seq[0]
    last = seq[cycles]
    assert (np.isnan(v[3]) and np.isnan(last)) or v[3] == last
    hist = v[4:]
    assert len(hist) == min(cycles, 64)
    np.testing.assert_array_equal(hist, np.array(seq[1:1 + len(hist)]))


def test_library_defines_every_internal_symbol():
    lib = os.path.join(ROOT, "paper_2607_10983_gb300", "_build", "libgbmg.so")
    nm = shutil.which("nm")
    if nm is None or not os.path.exists(lib):
        pytest.skip("nm or the built library is not available")
    out = subprocess.run([nm, "-C", "-u", lib], capture_output=True, text=True, check=True).stdout
    assert "gbmg::" not in out, out
