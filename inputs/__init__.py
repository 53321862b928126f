"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA library.

This module holds none of the multigrid method's arithmetic. It makes gauge
fields, sources and gauge transformations from counter-based random numbers
(Philox4x32-10, Salmon et al., SC'11) so that the oracle and the GPU path can be
fed bit-identical inputs. The heavy loops live in ``gen.c`` (plain C, OpenMP),
compiled in-tree with gcc on first use or by ``__graft_entry__.build()``.

Input recipe (the paper's gauge ensembles: quenched U(1), Wilson plaquette
action, periodic, beta = 6 and 10):
  * links: Metropolis from a cold start, ``sweeps`` sweeps, ``hits`` hits per link
    with proposals uniform in [-step, step] rad;
  * sources: complex Gaussian, Re and Im independent N(0, 1) (Box-Muller);
  * gauge transforms: uniform U(1) phases.

4d SU(3) recipe (Wilson-Dirac in four dimensions):
  * links: every U_x^mu the SU(3) projection of 1 + eps H (H Gaussian traceless
    hermitian, eps = 0.4), then ``ape_steps`` APE smearing steps with alpha = 0.5;
    the projection is row Gram-Schmidt with row 3 = conj(row 1 x row 2);
  * sources: complex Gaussian, 12 components (4 spins x 3 colours) per site.

Layouts: site x = x0 + L0*x1 (+ L0 L1 x2 + L0 L1 L2 x3 in 4d); links U[x, mu]
complex128 (U[x, mu, a, b] for SU(3)); spinors psi[x, s] complex128 (psi[x, s, c]
in 4d).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libmginputs.so")
_lock = threading.Lock()
_lib = None

# Root seed of every workload; each workload adds its own id (workload_seed mixes in L and beta).
ROOT_SEED = 20070704


def build(force: bool = False) -> str:
    """Compile gen.c into an in-tree shared library with gcc and return its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_GPU_SRC = os.path.join(_HERE, "metropolis_gpu.cu")
_GPU_LIB = os.path.join(_HERE, "libmginputs_gpu.so")
_gpu_lib = None


def build_gpu(force: bool = False) -> str:
    """Compile the GPU twin of the Metropolis generator (metropolis_gpu.cu) for sm_103a with nvcc."""
    if force or not os.path.exists(_GPU_LIB) or os.path.getmtime(_GPU_LIB) < os.path.getmtime(_GPU_SRC):
        import shutil
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = _GPU_LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-shared", "-Xcompiler",
               "-fPIC", "-o", tmp, _GPU_SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _GPU_LIB)
    return _GPU_LIB


def _load_gpu():
    global _gpu_lib
    with _lock:
        if _gpu_lib is None:
            lib = ctypes.CDLL(build_gpu())
            vp = ctypes.c_void_p
            lib.gen_metropolis_u1_2d_gpu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int, ctypes.c_double, vp, vp, vp, vp, vp]
            lib.gen_metropolis_u1_2d_gpu.restype = ctypes.c_int
            _gpu_lib = lib
    return _gpu_lib


def metropolis_u1_2d_gpu(L0: int, L1: int, betas, seeds, sweeps: int, hits: int = 10, step: float = 0.5):
    """The Markov chain of metropolis_u1_2d from a cold start, run on the current CUDA device for
    len(seeds) fields of L0 x L1 at once (beta and seed per field). Returns (theta[f, x, mu] on the
    host, acceptance per field). Check the result's digest against the CPU generator's where a
    stored digest exists: the two agree bit for bit unless an accept decision falls within the
    hosts' cos / sin / exp rounding difference."""
    import torch
    if L0 % 2 or L1 % 2:
        raise ValueError("Metropolis checkerboard needs even extents")
    nf = len(seeds)
    if len(betas) != nf:
        raise ValueError("one beta per seed")
    dev = torch.device("cuda", torch.cuda.current_device())
    theta = torch.zeros((nf, L0 * L1, 2), dtype=torch.float64, device=dev)
    b = torch.tensor([float(x) for x in betas], dtype=torch.float64, device=dev)
    sd = torch.tensor(np.array([int(x) for x in seeds], dtype=np.uint64).view(np.int64), device=dev)
    acc = torch.zeros(nf, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    rc = _load_gpu().gen_metropolis_u1_2d_gpu(L0, L1, nf, int(sweeps), int(hits), float(step), b.data_ptr(),
                                              sd.data_ptr(), theta.data_ptr(), acc.data_ptr(), stream.cuda_stream)
    if rc != 0:
        raise RuntimeError(f"GPU Metropolis generator: CUDA error {rc}")
    stream.synchronize()
    tot = max(1, sweeps * hits * 2 * L0 * L1)
    return theta.cpu().numpy(), (acc.cpu().numpy() / tot)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.gen_gaussian_complex.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, dp]
            lib.gen_uniform.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, dp]
            lib.metropolis_u1_2d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_uint64, dp, ctypes.POINTER(ctypes.c_int64)]
            lib.links_from_angles.argtypes = [ctypes.c_int64, dp, dp]
            lib.gen_u1_phases.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, dp]
            lib.gen_num_threads.restype = ctypes.c_int
            lib.gen_su3_near_identity.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, dp]
            lib.gen_su3_random.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, dp]
            lib.ape_smear_4d.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_double, dp, dp]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: four uint32 counter words, two uint32 key words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def gaussian_complex(n: int, seed: int, tag: int) -> np.ndarray:
    """n complex128 Gaussians (Re, Im ~ N(0,1)), Philox counter (i, tag), key seed."""
    out = np.empty(2 * n, dtype=np.float64)
    _load().gen_gaussian_complex(n, seed, tag, _dp(out))
    return out.view(np.complex128)


def uniform(n: int, seed: int, tag: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().gen_uniform(n, seed, tag, _dp(out))
    return out


def num_threads() -> int:
    return int(_load().gen_num_threads())


def metropolis_u1_2d(L0: int, L1: int, beta: float, sweeps: int, seed: int, hits: int = 10, step: float = 0.5,
                     theta0: np.ndarray | None = None):
    """Quenched U(1) link angles theta[x, mu] after ``sweeps`` Metropolis sweeps.

    Starts cold (theta = 0) unless ``theta0`` is given. Returns (theta, acceptance).
    """
    if L0 % 2 or L1 % 2:
        raise ValueError("Metropolis checkerboard needs even extents")
    theta = np.zeros((L0 * L1, 2), dtype=np.float64) if theta0 is None else np.array(theta0, dtype=np.float64)
    acc = ctypes.c_int64(0)
    _load().metropolis_u1_2d(L0, L1, float(beta), int(sweeps), int(hits), float(step), int(seed), _dp(theta),
                             ctypes.byref(acc))
    tot = max(1, sweeps * hits * 2 * L0 * L1)
    return theta, acc.value / tot


def links_from_angles(theta: np.ndarray) -> np.ndarray:
    th = np.ascontiguousarray(theta, dtype=np.float64)
    out = np.empty(2 * th.size, dtype=np.float64)
    _load().links_from_angles(th.size, _dp(th), _dp(out))
    return out.view(np.complex128).reshape(th.shape)


def u1_phases(nsites: int, seed: int, tag: int) -> np.ndarray:
    out = np.empty(2 * nsites, dtype=np.float64)
    _load().gen_u1_phases(nsites, seed, tag, _dp(out))
    return out.view(np.complex128)


def plaquette_angles(theta: np.ndarray, L0: int, L1: int) -> np.ndarray:
    """theta_p(x) = t0(x) + t1(x+0) - t0(x+1) - t1(x) wrapped to (-pi, pi], shape (L1, L0)."""
    t = theta.reshape(L1, L0, 2)
    tp = t[:, :, 0] + np.roll(t[:, :, 1], -1, axis=1) - np.roll(t[:, :, 0], -1, axis=0) - t[:, :, 1]
    w = np.remainder(tp + np.pi, 2 * np.pi) - np.pi
    w[w <= -np.pi] += 2 * np.pi
    return w


def topological_charge(theta: np.ndarray, L0: int, L1: int) -> float:
    """Q = (1/2pi) sum_x arg U_p(x), arg in (-pi, pi]; an integer up to rounding on a torus."""
    return float(plaquette_angles(theta, L0, L1).sum() / (2 * np.pi))


def field_digest(a: np.ndarray) -> str:
    """Short hash of an array's bytes (identifies a generated gauge field across hosts)."""
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:16]


# ---------------------------------------------------------------------------
# Workload recipes (seeds and sizes of the synthetic ensembles)
# ---------------------------------------------------------------------------

def workload_seed(workload_id: int, L: int, beta: float) -> int:
    """Seed of one gauge ensemble member: root seed + workload id, with L and beta mixed in."""
    return (ROOT_SEED + workload_id) * 1000003 + L * 101 + int(round(beta * 1000))


def member_seed(workload_id: int, L: int, beta: float, index: int) -> int:
    """Seed of member `index` of an ensemble of many fields (index 0 is workload_seed's field)."""
    return workload_seed(workload_id, L, beta) + (index << 40)


def schwinger_links_gpu(L: int, beta: float, sweeps: int = 2000, workload_id: int = 0, hits: int = 10,
                        step: float = 0.5, indices=(0,)):
    """Fields of the 2d U(1) ensemble recipe made by the GPU twin of the Metropolis chain:
    members `indices` (seed member_seed), links computed on the host from the angles exactly as
    schwinger_links does. Returns [(U, theta, acceptance)] per member."""
    seeds = [member_seed(workload_id, L, beta, i) for i in indices]
    th, acc = metropolis_u1_2d_gpu(L, L, [beta] * len(seeds), seeds, sweeps, hits=hits, step=step)
    return [(links_from_angles(th[k]), th[k], float(acc[k])) for k in range(len(seeds))]


def schwinger_links(L: int, beta: float, sweeps: int = 2000, workload_id: int = 0, hits: int = 10,
                    step: float = 0.5):
    """Gauge field U[x, mu] (complex128, (L*L, 2)) of the 2d U(1) ensemble recipe plus its angles."""
    seed = workload_seed(workload_id, L, beta)
    theta, acc = metropolis_u1_2d(L, L, beta, sweeps, seed, hits=hits, step=step)
    return links_from_angles(theta), theta, acc


def gaussian_source(L0: int, L1: int, seed: int, index: int = 0, ns: int = 2) -> np.ndarray:
    """Gaussian complex source chi[x, s] for right-hand side ``index``."""
    return gaussian_complex(L0 * L1 * ns, seed, 0x5352430000 + index).reshape(L0 * L1, ns)


def free_links(L0: int, L1: int, phi=(0.0, 0.0)) -> np.ndarray:
    """Constant U(1) links exp(i phi_mu) (phi = 0 is the free field)."""
    U = np.empty((L0 * L1, 2), dtype=np.complex128)
    U[:, 0] = np.exp(1j * phi[0])
    U[:, 1] = np.exp(1j * phi[1])
    return U


def hot_links(L0: int, L1: int, seed: int) -> np.ndarray:
    """Uniformly random U(1) links (infinite-temperature field)."""
    return u1_phases(L0 * L1 * 2, seed, 0x484F54).reshape(L0 * L1, 2)


# ---------------------------------------------------------------------------
# 4d SU(3)
# ---------------------------------------------------------------------------

def su3_near_identity(n: int, eps: float, seed: int, tag: int) -> np.ndarray:
    """n SU(3) matrices (n, 3, 3): projection of 1 + eps H, H Gaussian traceless hermitian."""
    out = np.empty(n * 18, dtype=np.float64)
    _load().gen_su3_near_identity(int(n), float(eps), int(seed), int(tag), _dp(out))
    return out.view(np.complex128).reshape(n, 3, 3)


def su3_random(n: int, seed: int, tag: int) -> np.ndarray:
    """n random SU(3) matrices (n, 3, 3): projection of complex Gaussian matrices."""
    out = np.empty(n * 18, dtype=np.float64)
    _load().gen_su3_random(int(n), int(seed), int(tag), _dp(out))
    return out.view(np.complex128).reshape(n, 3, 3)


def ape_smear(U: np.ndarray, dims, alpha: float = 0.5, steps: int = 1) -> np.ndarray:
    """``steps`` APE smearing steps of a 4d SU(3) field U[x, mu, a, b] (returns a new array)."""
    L = (ctypes.c_int * 4)(*[int(v) for v in dims])
    cur = np.ascontiguousarray(U, dtype=np.complex128).copy()
    nxt = np.empty_like(cur)
    for _ in range(int(steps)):
        _load().ape_smear_4d(L, float(alpha), _dp(cur.view(np.float64)), _dp(nxt.view(np.float64)))
        cur, nxt = nxt, cur
    return cur


def su3_links(dims, seed: int, eps: float = 0.4, ape_steps: int = 4, alpha: float = 0.5) -> np.ndarray:
    """4d SU(3) gauge field U[x, mu, a, b] (complex128, (V, 4, 3, 3)) of the recipe above."""
    V = int(np.prod(dims))
    U = su3_near_identity(V * 4, eps, seed, 0x535533).reshape(V, 4, 3, 3)
    return ape_smear(U, dims, alpha, ape_steps) if ape_steps > 0 else U


def gaussian_spinor(nsites: int, n_int: int, seed: int, index: int = 0) -> np.ndarray:
    """Gaussian complex field (nsites, n_int) for right-hand side ``index`` (any dimension)."""
    return gaussian_complex(nsites * n_int, seed, 0x5352430000 + index).reshape(nsites, n_int)
