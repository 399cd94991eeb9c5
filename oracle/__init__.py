"""CPU oracle for RANMAR (arXiv 2512.00093): test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.  The arithmetic lives in ``ranmar_oracle.c`` (plain C,
one routine per passage of the paper); this module builds it with gcc, loads
it with ctypes and wraps it for numpy arrays.  ``matrix.py`` adds the
companion-matrix form of Sec. 3.1 in plain numpy.

Every function states the passage it follows.  Parity is pinned (see
``tests/test_oracle_pins.py``) to: the published RANMAR test vector, the
equivalence of Algorithms 1 and 2, the equivalence of the integer and float
forms of Algorithm 3, brute-force stepping, Cayley-Hamilton on the matrix A,
the composition law, the exact multiplicative order of t modulo phi, and the
c-sequence closed form.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

R = 97
S = 33
MASK24 = 0xFFFFFF
M_C = (1 << 24) - 3
D_C = 7654321
C0 = 362436

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ranmar_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict[int, ctypes.CDLL] = {}

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32ref = ctypes.POINTER(ctypes.c_int32)
_u32ref = ctypes.POINTER(ctypes.c_uint32)
_f64ref = ctypes.POINTER(ctypes.c_double)


def lib_path(mutant: int = 0) -> str:
    name = "libranmar_oracle.so" if mutant == 0 else f"libranmar_oracle_m{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the C oracle with gcc (optionally with one planted mistake)."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           f"-DORC_MUTANT={mutant}", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    lib.orc_seed_int.argtypes = [ctypes.c_int32, _u32p]
    lib.orc_seed_int.restype = ctypes.c_int
    lib.orc_seed_float.argtypes = [ctypes.c_int32, _f64p]
    lib.orc_seed_float.restype = ctypes.c_int
    lib.orc_alg1.argtypes = [_f64p, _i32ref, _i32ref, _f64ref, ctypes.c_uint64, _f64p]
    lib.orc_alg1.restype = None
    lib.orc_alg2.argtypes = [_u32p, _i32ref, _i32ref, _u32ref, ctypes.c_uint64, ctypes.c_void_p]
    lib.orc_alg2.restype = None
    lib.orc_lammps_to_seq.argtypes = [_u32p, ctypes.c_int32, _u32p]
    lib.orc_lammps_to_seq.restype = None
    lib.orc_seq_to_lammps.argtypes = [_u32p, _u32p, _i32ref, _i32ref]
    lib.orc_seq_to_lammps.restype = None
    lib.orc_seeded_state.argtypes = [ctypes.c_int32, _u32p, _u32ref]
    lib.orc_seeded_state.restype = ctypes.c_int
    lib.orc_generate.argtypes = [_u32p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_generate.restype = None
    lib.orc_generate_alg1.argtypes = [_u32p, ctypes.c_uint32, ctypes.c_uint64, _f64p]
    lib.orc_generate_alg1.restype = None
    lib.orc_brute_jump.argtypes = [_u32p, _u32ref, ctypes.c_uint64]
    lib.orc_brute_jump.restype = None
    lib.orc_poly_mulmod.argtypes = [_u32p, _u32p, _u32p]
    lib.orc_poly_mulmod.restype = None
    lib.orc_poly_pow_t.argtypes = [_u32p, ctypes.c_int, _u32p]
    lib.orc_poly_pow_t.restype = None
    lib.orc_apply_dot.argtypes = [_u32p, _u32p, _u32p]
    lib.orc_apply_dot.restype = None
    lib.orc_apply_horner.argtypes = [_u32p, _u32p, _u32p]
    lib.orc_apply_horner.restype = None
    lib.orc_exp_mod_m.argtypes = [_u32p, ctypes.c_int]
    lib.orc_exp_mod_m.restype = ctypes.c_uint32
    lib.orc_c_jump.argtypes = [ctypes.c_uint32, _u32p, ctypes.c_int]
    lib.orc_c_jump.restype = ctypes.c_uint32
    lib.orc_c_step.argtypes = [ctypes.c_uint32, ctypes.c_uint64]
    lib.orc_c_step.restype = ctypes.c_uint32
    lib.orc_jump.argtypes = [_u32p, ctypes.c_uint32, _u32p, ctypes.c_int, _u32p, _u32ref]
    lib.orc_jump.restype = None
    lib.orc_stream.argtypes = [ctypes.c_int32, _u32p, ctypes.c_int, ctypes.c_uint64, _u32p]
    lib.orc_stream.restype = ctypes.c_int
    lib.orc_lfg_step.argtypes = [_u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
    lib.orc_lfg_step.restype = None
    lib.orc_lfg_mulmod.argtypes = [_u32p, _u32p, _u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int]
    lib.orc_lfg_mulmod.restype = None
    lib.orc_lfg_pow_t.argtypes = [_u32p, ctypes.c_int, _u32p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int]
    lib.orc_lfg_pow_t.restype = None
    lib.orc_lfg_apply.argtypes = [_u32p, _u32p, _u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.orc_lfg_apply.restype = None
    lib.orc_lfg_jump.argtypes = [_u32p, _u32p, ctypes.c_int, _u32p, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int]
    lib.orc_lfg_jump.restype = None
    lib.orc_lfg_generate.argtypes = [_u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_uint64, _u32p]
    lib.orc_lfg_generate.restype = None
    return lib


def load(mutant: int = 0) -> ctypes.CDLL:
    with _lock:
        if mutant not in _libs:
            _libs[mutant] = _declare(ctypes.CDLL(build(mutant)))
        return _libs[mutant]


class Oracle:
    """numpy-facing wrapper over one build of the C oracle."""

    def __init__(self, mutant: int = 0):
        self.lib = load(mutant)
        self.mutant = mutant

    # --- exponents ------------------------------------------------------
    @staticmethod
    def words(e: int, nw: int | None = None) -> np.ndarray:
        """Non-negative integer -> little-endian uint32 words."""
        if e < 0:
            raise ValueError("exponent must be non-negative")
        if nw is None:
            nw = max(1, (e.bit_length() + 31) // 32)
        if e >> (32 * nw):
            raise ValueError("exponent does not fit")
        return np.array([(e >> (32 * w)) & 0xFFFFFFFF for w in range(nw)], dtype=np.uint32)

    # --- Algorithm 3 ----------------------------------------------------
    def seed_int(self, seed: int) -> np.ndarray:
        u = np.zeros(R, np.uint32)
        if self.lib.orc_seed_int(seed, u) != 0:
            raise ValueError(f"seed {seed} outside 1..900000000")
        return u

    def seed_float(self, seed: int) -> np.ndarray:
        u = np.zeros(R, np.float64)
        if self.lib.orc_seed_float(seed, u) != 0:
            raise ValueError(f"seed {seed} outside 1..900000000")
        return u

    def seeded_state(self, seed: int) -> tuple[np.ndarray, int]:
        x = np.zeros(R, np.uint32)
        c = ctypes.c_uint32(0)
        if self.lib.orc_seeded_state(seed, x, ctypes.byref(c)) != 0:
            raise ValueError(f"seed {seed} outside 1..900000000")
        return x, c.value

    # --- Algorithms 1 and 2 on the LAMMPS ring ---------------------------
    def alg1(self, u: np.ndarray, i: int, j: int, c: float, n: int):
        u = np.ascontiguousarray(u, np.float64).copy()
        ii, jj, cc = ctypes.c_int32(i), ctypes.c_int32(j), ctypes.c_double(c)
        out = np.zeros(n, np.float64)
        self.lib.orc_alg1(u, ctypes.byref(ii), ctypes.byref(jj), ctypes.byref(cc), n, out)
        return out, (u, ii.value, jj.value, cc.value)

    def alg2(self, u: np.ndarray, i: int, j: int, v: int, n: int):
        u = np.ascontiguousarray(u, np.uint32).copy()
        ii, jj, vv = ctypes.c_int32(i), ctypes.c_int32(j), ctypes.c_uint32(v)
        out = np.zeros(n, np.uint32)
        self.lib.orc_alg2(u, ctypes.byref(ii), ctypes.byref(jj), ctypes.byref(vv), n,
                          out.ctypes.data if n else None)
        return out, (u, ii.value, jj.value, vv.value)

    def lammps_to_seq(self, u: np.ndarray, i: int) -> np.ndarray:
        x = np.zeros(R, np.uint32)
        self.lib.orc_lammps_to_seq(np.ascontiguousarray(u, np.uint32), i, x)
        return x

    def seq_to_lammps(self, x: np.ndarray):
        u = np.zeros(R, np.uint32)
        ii, jj = ctypes.c_int32(0), ctypes.c_int32(0)
        self.lib.orc_seq_to_lammps(np.ascontiguousarray(x, np.uint32), u, ctypes.byref(ii),
                                   ctypes.byref(jj))
        return u, ii.value, jj.value

    # --- sequence-order state --------------------------------------------
    def generate(self, x: np.ndarray, c: int, n: int):
        """n 24-bit outputs (Algorithm 2) and the advanced state."""
        x = np.ascontiguousarray(x, np.uint32)
        out = np.zeros(n, np.uint32)
        xa = np.zeros(R, np.uint32)
        ca = ctypes.c_uint32(0)
        self.lib.orc_generate(x, c, n, out.ctypes.data if n else None, xa.ctypes.data,
                              ctypes.addressof(ca))
        return out, xa, ca.value

    def generate_alg1(self, x: np.ndarray, c: int, n: int) -> np.ndarray:
        """n outputs of the same stream through Algorithm 1 in double."""
        out = np.zeros(n, np.float64)
        self.lib.orc_generate_alg1(np.ascontiguousarray(x, np.uint32), c, n, out)
        return out

    def brute_jump(self, x: np.ndarray, c: int, J: int):
        x = np.ascontiguousarray(x, np.uint32).copy()
        cc = ctypes.c_uint32(c)
        self.lib.orc_brute_jump(x, ctypes.byref(cc), J)
        return x, cc.value

    # --- Sec. 3.1 / 3.2 ---------------------------------------------------
    def poly_mulmod(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        out = np.zeros(R, np.uint32)
        self.lib.orc_poly_mulmod(np.ascontiguousarray(a, np.uint32),
                                 np.ascontiguousarray(b, np.uint32), out)
        return out

    def poly_pow_t(self, e: int) -> np.ndarray:
        w = self.words(e)
        out = np.zeros(R, np.uint32)
        self.lib.orc_poly_pow_t(w, len(w), out)
        return out

    def apply_dot(self, x: np.ndarray, b: np.ndarray) -> np.ndarray:
        out = np.zeros(R, np.uint32)
        self.lib.orc_apply_dot(np.ascontiguousarray(x, np.uint32),
                               np.ascontiguousarray(b, np.uint32), out)
        return out

    def apply_horner(self, x: np.ndarray, b: np.ndarray) -> np.ndarray:
        out = np.zeros(R, np.uint32)
        self.lib.orc_apply_horner(np.ascontiguousarray(x, np.uint32),
                                  np.ascontiguousarray(b, np.uint32), out)
        return out

    def exp_mod_m(self, e: int) -> int:
        w = self.words(e)
        return int(self.lib.orc_exp_mod_m(w, len(w)))

    def c_jump(self, c: int, e: int) -> int:
        w = self.words(e)
        return int(self.lib.orc_c_jump(c, w, len(w)))

    def c_step(self, c: int, n: int) -> int:
        return int(self.lib.orc_c_step(c, n))

    def jump(self, x: np.ndarray, c: int, e: int):
        w = self.words(e)
        xo = np.zeros(R, np.uint32)
        co = ctypes.c_uint32(0)
        self.lib.orc_jump(np.ascontiguousarray(x, np.uint32), c, w, len(w), xo, ctypes.byref(co))
        return xo, co.value

    def stream(self, seed: int, e: int, count: int) -> np.ndarray:
        """First `count` outputs of the block that starts e transitions after
        the seeded state (stream k of (seed, J) has e = k*J, Sec. 1)."""
        w = self.words(e)
        out = np.zeros(count, np.uint32)
        if self.lib.orc_stream(seed, w, len(w), count, out) != 0:
            raise ValueError(f"seed {seed} outside 1..900000000")
        return out

    # -- general lags (concluding remarks): x_n = x_{n-r} - x_{n-s} mod 2^e --
    def lfg_step(self, x: np.ndarray, r: int, s: int, e: int, n: int) -> np.ndarray:
        """n transitions of the window x (oldest first), brute force."""
        y = np.ascontiguousarray(x, np.uint32).copy()
        self.lib.orc_lfg_step(y, r, s, e, n)
        return y

    def lfg_mulmod(self, a, b, r: int, s: int, e: int, karatsuba: bool = False) -> np.ndarray:
        """a b mod phi_{r,s} = t^r + t^{r-s} - 1 (classical or Karatsuba product)."""
        out = np.zeros(r, np.uint32)
        self.lib.orc_lfg_mulmod(np.ascontiguousarray(a, np.uint32), np.ascontiguousarray(b, np.uint32),
                                out, r, s, e, int(karatsuba))
        return out

    def lfg_pow_t(self, E: int, r: int, s: int, e: int, karatsuba: bool = False) -> np.ndarray:
        """t^E mod phi_{r,s} by left-to-right binary exponentiation."""
        w = self.words(E)
        out = np.zeros(r, np.uint32)
        self.lib.orc_lfg_pow_t(w, len(w), out, r, s, e, int(karatsuba))
        return out

    def lfg_apply(self, x, p, r: int, s: int, e: int) -> np.ndarray:
        """x P(A) in the dot-product form (window extended to 2r - 1 words)."""
        out = np.zeros(r, np.uint32)
        self.lib.orc_lfg_apply(np.ascontiguousarray(x, np.uint32), np.ascontiguousarray(p, np.uint32),
                               out, r, s, e)
        return out

    def lfg_generate(self, x, r: int, s: int, e: int, n: int):
        """(the next n words of the recurrence, the advanced window)."""
        y = np.ascontiguousarray(x, np.uint32).copy()
        out = np.zeros(max(n, 1), np.uint32)
        self.lib.orc_lfg_generate(y, r, s, e, n, out)
        return out[:n], y

    def lfg_jump(self, x, E: int, r: int, s: int, e: int, karatsuba: bool = False) -> np.ndarray:
        """The window x jumped by E transitions (polynomial method)."""
        w = self.words(E)
        out = np.zeros(r, np.uint32)
        self.lib.orc_lfg_jump(np.ascontiguousarray(x, np.uint32), w, len(w), out, r, s, e,
                              int(karatsuba))
        return out


_default: Oracle | None = None


def oracle() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(0)
    return _default
