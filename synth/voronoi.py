"""Seeded clipped-Voronoi / CVT meshes of the unit cube (host C++ generator).

``voronoi_mesh(n, seed, lloyd)`` draws n seeds uniformly in [0,1]^3 with
numpy's PCG64 (``default_rng(seed)``), runs ``lloyd`` Lloyd iterations (each
seed moved to its cell's barycentre) and returns the clipped Voronoi
diagram as a face-based ``Mesh``.  The face between cells i < j is stored
once, oriented from i to j; boundary faces (flag 1) point out of the cube.
The generator (voronoi.cpp) is compiled on first use with g++ -fopenmp.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from .meshes import Mesh

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "voronoi.cpp")
_LIB = os.path.join(_DIR, "_lib", "libvoronoi.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".tmp"
        subprocess.run(["g++", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c++17", _SRC, "-o", tmp],
                       check=True, capture_output=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.voronoi_build.restype = C.c_void_p
        L.voronoi_build.argtypes = [C.c_int64, C.c_void_p, C.c_int]
        L.voronoi_sizes.argtypes = [C.c_void_p] + [C.POINTER(C.c_int64)] * 6
        L.voronoi_copy.argtypes = [C.c_void_p] + [C.c_void_p] * 6
        L.voronoi_free.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def voronoi_mesh(n: int, seed: int = 0, lloyd: int = 10, bc: int = 1, return_seeds: bool = False):
    L = _load()
    rng = np.random.default_rng(seed)
    seeds = np.ascontiguousarray(rng.uniform(0.0, 1.0, size=(n, 3)))
    r = L.voronoi_build(n, seeds.ctypes.data, lloyd)
    sz = [C.c_int64() for _ in range(6)]
    L.voronoi_sizes(r, *[C.byref(x) for x in sz])
    nv, nf, nfv, nc, ncf, dropped = [x.value for x in sz]
    xyz = np.zeros((nv, 3))
    fptr = np.zeros(nf + 1, dtype=np.int64)
    fv = np.zeros(nfv, dtype=np.int32)
    cptr = np.zeros(nc + 1, dtype=np.int64)
    cf = np.zeros(ncf, dtype=np.int32)
    fbc = np.zeros(nf, dtype=np.int8)
    L.voronoi_copy(r, xyz.ctypes.data, fptr.ctypes.data, fv.ctypes.data, cptr.ctypes.data,
                   cf.ctypes.data, fbc.ctypes.data)
    L.voronoi_free(r)
    fbc[fbc != 0] = bc
    mesh = Mesh(xyz, fptr, fv, cptr, cf, fbc, name=f"voronoi{n}_s{seed}_l{lloyd}")
    mesh.dropped_faces = int(dropped)
    if return_seeds:
        return mesh, seeds
    return mesh
