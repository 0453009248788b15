"""Orbit averaging of element fields under the cube's symmetry groups (FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. 6.1: a symmetry type splits the cell into orbits of elements, and enforcing it sets
every density (and, in the loop of Sec. 5.2, every sensitivity) on an orbit to the
orbit's average. Three types:

* reflect3 - reflections in the three mid-planes x = 1/2, y = 1/2, z = 1/2 (8 maps);
* rotate3  - the rotations of the cube about its centre generated by quarter turns about
             the three axes (24 maps: the proper signed permutations of the axes);
* reflect6 - the mid-plane reflections together with the reflections in the diagonal
             planes through the centre; the printed plane equations "x+y=0" etc. are
             read as the planes x = y, y = z, z = x (the other reading puts them outside
             the cell), which together generate all 48 signed permutations.

Each map is a signed permutation of the axes acting on element centres relative to the
cell centre. The average over the group's images of an element equals the average over
its orbit (every orbit member appears |stabiliser| times).
"""
from __future__ import annotations

import itertools

import numpy as np

KINDS = ("reflect3", "rotate3", "reflect6")


def _perm_parity(p) -> int:
    inv = sum(1 for a in range(3) for b in range(a + 1, 3) if p[a] > p[b])
    return -1 if inv % 2 else 1


def group(kind: str):
    """List of (perm, flips): the image of element index (i0, i1, i2) has index
    j_k = i_perm[k], replaced by n-1-j_k where flips[k]."""
    maps = []
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((False, True), repeat=3):
            det = _perm_parity(perm) * (-1) ** sum(flips)
            if kind == "reflect3" and perm != (0, 1, 2):
                continue
            if kind == "rotate3" and det != 1:
                continue
            if kind not in KINDS:
                raise ValueError(kind)
            maps.append((perm, flips))
    return maps


def image_index(idx, perm, flips, n):
    """Index triple (x, y, z) of the image of element (x, y, z)."""
    out = []
    for k in range(3):
        j = idx[perm[k]]
        out.append(n - 1 - j if flips[k] else j)
    return tuple(out)


def symmetrize(field: np.ndarray, n: int, kind: str) -> np.ndarray:
    """Average over the group's images of every element. field: n^3 values, x fastest."""
    A = np.asarray(field, dtype=np.float64).reshape(n, n, n)     # [z, y, x]
    acc = np.zeros_like(A)
    G = group(kind)
    # element (x, y, z) = A[z, y, x]; axis k of (x, y, z) is array axis 2 - k
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    idx = (xx, yy, zz)
    for perm, flips in G:
        j = [idx[perm[k]] for k in range(3)]
        j = [n - 1 - j[k] if flips[k] else j[k] for k in range(3)]
        acc += A[j[2], j[1], j[0]]
    return (acc / len(G)).ravel()
