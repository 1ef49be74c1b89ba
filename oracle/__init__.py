"""CPU oracle for Frobenius inversion -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_2208_01239_gb300``) never imports, links or runs it, and
it shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (plain C, FP64, compiled with gcc and
``-ffp-contract=off`` so that x86 and Arm hosts round identically).  This
module only marshals numpy arrays into it.  Each routine follows one algorithm
of Dai, Lim and Ye, "Complex matrix inversion via real matrix inversions":

* :func:`cplx_lu_inv`   -- Algorithm "Inversion with LU decomposition" (Sec. 4)
                           and its right-inverse variant.
* :func:`cplx_chol_inv` -- Algorithm "Inversion with Cholesky decomposition"
                           (Sec. 4.3).
* :func:`frob_inv_basic` -- Algorithm "Frobenius inversion" with tau = 1
                           (Sec. 2, Lemma 2.3): two explicit real inversions,
                           three products, one addition.
* :func:`frob_inv_b`    -- the formula for invertible B (Sec. 4.2, before
                           Lemma "rand Frob"), explicit real inversions.
* :func:`bicomplex_inv` -- inverse of a bicomplex matrix A + jB (Sec. 2.4,
                           m = 2) through its 2n complex embedding.
* :func:`frob_inv_lu`   -- Algorithm "Frobenius inversion with LU
                           decomposition" (Sec. 4.1).
* :func:`frob_inv_rand` -- Algorithm "Almost sure Frobenius inversion"
                           (Sec. 4.2), with mu supplied by the caller.
* :func:`frob_inv_chol` -- Algorithm "Frobenius inversion with Cholesky
                           decomposition" (Sec. 4.3).
* :func:`inv2x2`, :func:`adjugate_inv` -- closed forms used as pins.
* :func:`inv_adjoint`   -- -X^H G X^H, the gradient of a real loss through
                           X = M^{-1} (from d(M^{-1}) = -M^{-1} dM M^{-1}).
* :func:`frob_solve`    -- Algorithm "Linear system with Frobenius
                           inversion" (Sec. 3), several right-hand sides.
* :func:`sign_newton`   -- Newton's iteration for the matrix sign function
                           (Sec. 5.3, eq. "iter"), fixed step count.
* :func:`newton`        -- the same iteration, or the polar one (Sec. 5.5,
                           eq. "iter2"), with the stopping rule of Sec. 5.3.
* :func:`sylvester`     -- Sylvester equation by the sign of a block matrix
                           (Sec. 5.4); Lyapunov with B = A^H.
* :func:`polar`         -- polar decomposition X = Q P (Sec. 5.5).

Every function is pinned by ``tests/test_oracle_*.py`` against values fixed by
mathematics (closed forms, brute force, identities from the paper, LAPACK via
numpy on special cases); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_instances: dict = {}


def _so_path(mutant: int) -> str:
    return os.path.join(_BUILD_DIR, "liboracle.so" if mutant == 0 else f"liboracle_mut{mutant}.so")


def build(force: bool = False, mutant: int = 0) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` with gcc (OpenMP if
    available).  ``mutant`` > 0 builds a copy with one planted mistake, for the
    test that checks the pins catch it.  Returns the library path."""
    so = _so_path(mutant)
    with _lock:
        if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(_SRC):
            return so
        os.makedirs(_BUILD_DIR, exist_ok=True)
        cc = os.environ.get("CC", shutil.which("gcc") or "cc")
        tmp = f"{so}.{os.getpid()}.tmp"
        base = [cc, "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", f"-DORC_MUTANT={int(mutant)}",
                _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, so)
        return so


class OracleError(RuntimeError):
    """A factorisation met an exactly zero / non-finite pivot (LU) or a
    non-positive diagonal (Cholesky).  ``info`` is the LAPACK-style 1-based
    index of the failing step."""

    def __init__(self, what: str, info: int):
        super().__init__(f"{what}: info={info}")
        self.info = info


def _prep(m) -> tuple[np.ndarray, int]:
    m = np.ascontiguousarray(np.asarray(m, dtype=np.complex128))
    if m.ndim != 2 or m.shape[0] != m.shape[1]:
        raise ValueError("expected a square matrix")
    return m, m.shape[0]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(what: str, info: int):
    if info != 0:
        raise OracleError(what, info)


class Oracle:
    """The oracle routines bound to one compiled copy of ``oracle.c``."""

    def __init__(self, so_path: str):
        lib = ctypes.CDLL(so_path)
        zp = ctypes.c_void_p
        i = ctypes.c_int
        sig = {
            "orc_cplx_lu_inv": [i, zp, zp, i],
            "orc_cplx_chol_inv": [i, zp, zp],
            "orc_frob_inv_basic": [i, zp, zp, zp, zp, zp],
            "orc_frob_inv_lu": [i, zp, zp],
            "orc_frob_inv_b": [i, zp, zp],
            "orc_bicomplex_inv": [i, zp, zp, zp, zp],
            "orc_frob_inv_rand": [i, zp, ctypes.c_double, zp],
            "orc_frob_inv_chol": [i, zp, zp],
            "orc_inv2x2": [zp, zp],
            "orc_adjugate_inv": [i, zp, zp],
            "orc_num_threads": [],
            "orc_inv_adjoint": [i, zp, zp, zp],
            "orc_sign_newton": [i, zp, i, zp],
            "orc_frob_solve": [i, i, zp, zp, zp],
            "orc_newton": [i, zp, i, ctypes.c_double, i, zp, zp],
            "orc_sylvester": [i, i, zp, zp, zp, ctypes.c_double, i, zp, zp],
            "orc_polar": [i, zp, ctypes.c_double, i, zp, zp, zp],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        self.lib = lib

    def cplx_lu_inv(self, m, left: bool = False) -> np.ndarray:
        """Complex LU inversion with partial pivoting (left=True: the paper's
        U X1 = I, X2 L = X1, X2 P order; left=False: the right inverse)."""
        m, n = _prep(m)
        x = np.empty_like(m)
        _check("cplx_lu_inv", self.lib.orc_cplx_lu_inv(n, _ptr(m), _ptr(x), int(left)))
        return x

    def cplx_chol_inv(self, m) -> np.ndarray:
        """Complex Cholesky inversion of a Hermitian positive definite matrix
        (lower triangle read)."""
        m, n = _prep(m)
        x = np.empty_like(m)
        _check("cplx_chol_inv", self.lib.orc_cplx_chol_inv(n, _ptr(m), _ptr(x)))
        return x

    def frob_inv_basic(self, m, stages: bool = False):
        """Frobenius inversion with explicit real inversions.  With
        ``stages=True`` also returns (A^{-1}B, S, S^{-1})."""
        m, n = _prep(m)
        x = np.empty_like(m)
        x2 = np.empty((n, n))
        s = np.empty((n, n))
        sinv = np.empty((n, n))
        _check("frob_inv_basic",
               self.lib.orc_frob_inv_basic(n, _ptr(m), _ptr(x), _ptr(x2), _ptr(s), _ptr(sinv)))
        return (x, (x2, s, sinv)) if stages else x

    def frob_inv_b(self, m) -> np.ndarray:
        """The formula for invertible B (Sec. 4.2): B^{-1}A(AB^{-1}A + B)^{-1}
        - i(AB^{-1}A + B)^{-1}, explicit real inversions."""
        m, n = _prep(m)
        x = np.empty_like(m)
        _check("frob_inv_b", self.lib.orc_frob_inv_b(n, _ptr(m), _ptr(x)))
        return x

    def bicomplex_inv(self, a, b):
        """(A + jB)^{-1} = Y0 + jY1 for bicomplex matrices (j^2 = -1, j
        commuting with i; the m = 2 iterated quadratic extension of Sec. 2.4),
        from the inverse of the embedding [[A, -B], [B, A]].  Returns (Y0, Y1)."""
        a, n = _prep(a)
        b = np.ascontiguousarray(np.asarray(b, dtype=np.complex128))
        if b.shape != (n, n):
            raise ValueError("A and B must both be n x n")
        y0 = np.empty_like(a)
        y1 = np.empty_like(a)
        _check("bicomplex_inv", self.lib.orc_bicomplex_inv(n, _ptr(a), _ptr(b), _ptr(y0), _ptr(y1)))
        return y0, y1

    def frob_inv_lu(self, m) -> np.ndarray:
        m, n = _prep(m)
        x = np.empty_like(m)
        _check("frob_inv_lu", self.lib.orc_frob_inv_lu(n, _ptr(m), _ptr(x)))
        return x

    def frob_inv_rand(self, m, mu: float) -> np.ndarray:
        m, n = _prep(m)
        x = np.empty_like(m)
        _check("frob_inv_rand", self.lib.orc_frob_inv_rand(n, _ptr(m), float(mu), _ptr(x)))
        return x

    def frob_inv_chol(self, m) -> np.ndarray:
        """Frobenius inversion with two real Cholesky factorisations; reads the
        lower triangle of the Hermitian input.  info in 1..n: A not positive
        definite; info in n+1..2n: S not positive definite."""
        m, n = _prep(m)
        x = np.empty_like(m)
        _check("frob_inv_chol", self.lib.orc_frob_inv_chol(n, _ptr(m), _ptr(x)))
        return x

    def inv2x2(self, m) -> np.ndarray:
        m, n = _prep(m)
        if n != 2:
            raise ValueError("inv2x2 needs a 2x2 matrix")
        x = np.empty_like(m)
        _check("inv2x2", self.lib.orc_inv2x2(_ptr(m), _ptr(x)))
        return x

    def adjugate_inv(self, m) -> np.ndarray:
        """adj(M)/det(M) by Laplace expansion, n <= 4."""
        m, n = _prep(m)
        x = np.empty_like(m)
        _check("adjugate_inv", self.lib.orc_adjugate_inv(n, _ptr(m), _ptr(x)))
        return x

    def num_threads(self) -> int:
        """OpenMP threads the oracle uses (1 if built without OpenMP)."""
        return int(self.lib.orc_num_threads())

    def inv_adjoint(self, x, g) -> np.ndarray:
        """-X^H G X^H: the gradient with respect to M of a real loss whose
        gradient with respect to X = M^{-1} is G."""
        x, n = _prep(x)
        g, n2 = _prep(g)
        if n != n2:
            raise ValueError("shape mismatch")
        out = np.empty_like(x)
        _check("inv_adjoint", self.lib.orc_inv_adjoint(n, _ptr(x), _ptr(g), _ptr(out)))
        return out

    def frob_solve(self, m, rhs) -> np.ndarray:
        """Solve M X = RHS (RHS n x nrhs complex) by Algorithm "Linear system
        with Frobenius inversion" (Sec. 3)."""
        m, n = _prep(m)
        rhs = np.ascontiguousarray(np.asarray(rhs, dtype=np.complex128))
        vec = rhs.ndim == 1
        r2 = rhs.reshape(n, -1).copy()
        x = np.empty_like(r2)
        _check("frob_solve", self.lib.orc_frob_solve(n, r2.shape[1], _ptr(m), _ptr(r2), _ptr(x)))
        return x[:, 0] if vec else x

    def sign_newton(self, m, iters: int) -> np.ndarray:
        """`iters` Newton steps X <- (X + X^{-1})/2 from X = M (Sec. 5.3)."""
        m, n = _prep(m)
        out = np.empty_like(m)
        _check("sign_newton", self.lib.orc_sign_newton(n, _ptr(m), int(iters), _ptr(out)))
        return out

    def newton(self, m, variant: int, eps: float, kmax: int):
        """Newton's iteration with the stopping rule of Sec. 5.3: variant 0
        X <- (X + X^{-1})/2 (sign), variant 1 X <- (X + X^{-H})/2 (polar
        factor).  Returns (X, steps)."""
        m, n = _prep(m)
        out = np.empty_like(m)
        steps = ctypes.c_int(0)
        _check("newton", self.lib.orc_newton(n, _ptr(m), int(variant), float(eps), int(kmax), _ptr(out),
                                             ctypes.byref(steps)))
        return out, steps.value

    def sylvester(self, a, b, c, eps: float, kmax: int):
        """Y with A Y + Y B = C through the sign of [[A, -C], [0, -B]]
        (Sec. 5.4).  Returns (Y, steps)."""
        a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
        b = np.ascontiguousarray(np.asarray(b, dtype=np.complex128))
        c = np.ascontiguousarray(np.asarray(c, dtype=np.complex128))
        p, q = a.shape[0], b.shape[0]
        if a.shape != (p, p) or b.shape != (q, q) or c.shape != (p, q):
            raise ValueError("shapes: A p x p, B q x q, C p x q")
        y = np.empty((p, q), dtype=np.complex128)
        steps = ctypes.c_int(0)
        _check("sylvester", self.lib.orc_sylvester(p, q, _ptr(a), _ptr(b), _ptr(c), float(eps), int(kmax), _ptr(y),
                                                   ctypes.byref(steps)))
        return y, steps.value

    def polar(self, x, eps: float, kmax: int):
        """X = Q P (Sec. 5.5): Q by Newton's iteration X <- (X + X^{-H})/2,
        P = Q^H X.  Returns (Q, P, steps)."""
        x, n = _prep(x)
        q = np.empty_like(x)
        pm = np.empty_like(x)
        steps = ctypes.c_int(0)
        _check("polar", self.lib.orc_polar(n, _ptr(x), float(eps), int(kmax), _ptr(q), _ptr(pm), ctypes.byref(steps)))
        return q, pm, steps.value


def load(mutant: int = 0) -> Oracle:
    """The oracle bound to the normal build (mutant=0) or a planted-mistake
    build (mutant=k)."""
    if mutant not in _instances:
        _instances[mutant] = Oracle(build(mutant=mutant))
    return _instances[mutant]


def cplx_lu_inv(m, left: bool = False):
    return load().cplx_lu_inv(m, left)


def cplx_chol_inv(m):
    return load().cplx_chol_inv(m)


def frob_inv_basic(m, stages: bool = False):
    return load().frob_inv_basic(m, stages)


def frob_inv_b(m):
    return load().frob_inv_b(m)


def bicomplex_inv(a, b):
    return load().bicomplex_inv(a, b)


def frob_inv_lu(m):
    return load().frob_inv_lu(m)


def frob_inv_rand(m, mu: float):
    return load().frob_inv_rand(m, mu)


def frob_inv_chol(m):
    return load().frob_inv_chol(m)


def inv2x2(m):
    return load().inv2x2(m)


def adjugate_inv(m):
    return load().adjugate_inv(m)


def num_threads() -> int:
    return load().num_threads()


def inv_adjoint(x, g):
    return load().inv_adjoint(x, g)


def sign_newton(m, iters: int):
    return load().sign_newton(m, iters)


def newton(m, variant: int, eps: float, kmax: int):
    return load().newton(m, variant, eps, kmax)


def sylvester(a, b, c, eps: float, kmax: int):
    return load().sylvester(a, b, c, eps, kmax)


def polar(x, eps: float, kmax: int):
    return load().polar(x, eps, kmax)


def frob_solve(m, rhs):
    return load().frob_solve(m, rhs)


from . import metrics  # noqa: E402,F401
