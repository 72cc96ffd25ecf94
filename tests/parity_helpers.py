"""Helpers of the GPU parity tests (no tests here).

FP32 arithmetic maps the nodes of moving spheres from FP32 centres, whose
last bits also vary from run to run with the summation order of the link
forces, so a node lying within that rounding of a mapped sphere's surface
can be covered or uncovered one step apart on the GPU and in the FP64
oracle.  Such a node changes the populations around it by ~1e-4; the
comparisons below record every disagreement of the node maps, require it
to be rare and to lie on a mapped surface, and exclude the nodes the
difference can reach.
"""
import numpy as np

import oracle as O
from paper_1904_02929_gb300 import susp as S


def dilate(m):
    out = m.copy()
    for ax in range(3):
        for sft in (-1, 1):
            out |= np.roll(m, sft, axis=ax)
    return out


def fp32_particle_pop_err(g, o, steps, radius, a_map_ratio=0.95, **sh):
    """Step the GPU machine g and the oracle o together one step at a time and
    return the population error (max |g - o| over max |o|) over the nodes
    fluid on both sides and out of reach of any node-map disagreement."""
    nz, ny, nx = g.owner().shape
    box = np.array([nx, ny, nz])
    ever = np.zeros((nz, ny, nx), bool)
    for _ in range(steps):
        g.step(1, S.make_shear(**sh))
        o.step(1, O.shear(**sh))
        og, oo = g.owner(), o.owner()
        diff = og != oo
        ever |= diff
        assert diff.mean() < 1e-4
        Ro, _, _ = o.particles()
        for z, y, x in np.argwhere(diff):
            i = max(og[z, y, x], oo[z, y, x])
            d = np.array([x, y, z], dtype=float) - Ro[i]
            d -= box * np.round(d / box)
            assert abs(np.linalg.norm(d) - a_map_ratio * radius[i]) < 1e-3
    near = ever
    for _ in range(steps):
        near = dilate(near)
    keep = ~near & (og < 0) & (oo < 0)
    fo, fg = o.populations(), g.populations()
    return np.abs(fg[:, keep] - fo[:, keep]).max() / np.abs(fo[:, keep]).max()
