"""Helpers of the GPU parity tests (no tests here).

FP32 arithmetic gives particle forces, and so centres, that differ from the
FP64 oracle's in the last bits (and, through the summation order of the link
forces, from run to run), so a node lying within that difference of a mapped
sphere's surface can be covered or uncovered one step apart on the GPU and
in the oracle.  (The node maps of every path take the solid / fluid
decision of nodes near a surface in FP64, so such flips need the centres
themselves to differ by the node's distance from the surface.)  A flip
gives the node its equilibrium populations one step early or late, which
changes them by the node's density deviation and non-equilibrium part: up
to a few 1e-4 of the largest population next to a sheared surface (one
flip in Ladd's FP32 run left 2.0e-4; the oracle against itself with every
centre moved by 1e-5 left at most 1.4e-5).  The comparison below therefore steps both sides together, checks
that every node-map disagreement lies on a mapped surface within the
distance the two sides' centres differ by, measures the population error
at every step while the two node maps have agreed throughout, and the
error at the end.
"""
from dataclasses import dataclass

import numpy as np

import oracle as O
from paper_1904_02929_gb300 import susp as S

# population error allowed after node-map flips (a fraction of the largest
# population): the order of a flipped node's non-equilibrium part
FLIP_TOL = 1e-3


def dilate(m):
    out = m.copy()
    for ax in range(3):
        for sft in (-1, 1):
            out |= np.roll(m, sft, axis=ax)
    return out


@dataclass
class Comparison:
    err_agree: float    # largest population error over the steps before the first flip
    steps_agree: int    # steps before the first node-map disagreement
    err_end: float      # population error after the last step
    flips: int          # node-map disagreements counted over all steps

    def check(self, pop_tol):
        """The error before the first flip, and the final one if no flip
        happened, within pop_tol; after a flip the final error within the
        change a flip makes."""
        if self.steps_agree > 0:
            assert self.err_agree < pop_tol, self
        assert self.err_end < (pop_tol if self.flips == 0 else max(pop_tol, FLIP_TOL)), self
        return self


def _pop_err(g, o):
    og, oo = g.owner(), o.owner()
    keep = (og < 0) & (oo < 0)
    fo, fg = o.populations(), g.populations()
    return float(np.abs(fg[:, keep] - fo[:, keep]).max() / np.abs(fo[:, keep]).max())


def _surface_gap(x, centre, a_map, box, delta):
    """Smallest | |x - image of centre| - a_map | over the periodic images,
    with the x shift of +-delta of the images across the Lees-Edwards planes
    y = 0 / L_y (either sign: the check only bounds the distance)."""
    best = np.inf
    for ky in (-1, 0, 1):
        for sgn in (1.0, -1.0):
            d = np.asarray(x, float) - centre
            d[1] += ky * box[1]
            d[0] += sgn * ky * delta
            d[0] -= box[0] * np.round(d[0] / box[0])
            d[2] -= box[2] * np.round(d[2] / box[2])
            best = min(best, abs(np.linalg.norm(d) - a_map))
    return best


def fp32_particle_comparison(g, o, steps, radius, a_map_ratio=0.95, **sh):
    """Step the GPU machine g and the oracle o together one step at a time;
    return a Comparison (populations over the nodes fluid on both sides,
    errors as max |g - o| over max |o|).  The node maps are compared from
    the start, before the first step."""
    nz, ny, nx = g.owner().shape
    box = np.array([nx, ny, nz], float)
    a_map = a_map_ratio * np.asarray(radius, float)
    err_agree, steps_agree, flips, agree = 0.0, 0, 0, True
    prev = None
    for step in range(steps + 1):
        if step > 0:
            g.step(1, S.make_shear(**sh))
            o.step(1, O.shear(**sh))
        Rg, _, _ = g.particles()
        Ro, _, _ = o.particles()
        cur = (Rg, Ro, o.delta)
        Rg0, Ro0, delta0 = prev if prev is not None else cur
        og, oo = g.owner(), o.owner()
        diff = og != oo
        if diff.any():
            agree = False
            flips += int(diff.sum())
            # the maps may come from the centres before or after the step,
            # and FP32 distances round at ~1e-5 of a lattice unit
            dR = np.maximum(np.linalg.norm(Rg - Ro, axis=1), np.linalg.norm(Rg0 - Ro0, axis=1)) + 1e-5
            for z, y, x in np.argwhere(diff):
                i = max(og[z, y, x], oo[z, y, x])
                gap = min(_surface_gap((x, y, z), c, a_map[i], box, dl)
                          for c in (Ro[i], Ro0[i]) for dl in (o.delta, delta0))
                assert gap <= dR[i], (step, x, y, z, i, gap, dR[i])
        if agree and step > 0:
            err_agree = max(err_agree, _pop_err(g, o))
            steps_agree += 1
        prev = cur
    return Comparison(err_agree, steps_agree, _pop_err(g, o), flips)


def fp32_particle_pop_err(g, o, steps, radius, pop_tol, a_map_ratio=0.95, **sh):
    """fp32_particle_comparison, checked against pop_tol and printed; returns
    the final population error."""
    c = fp32_particle_comparison(g, o, steps, radius, a_map_ratio, **sh)
    print(c)
    return c.check(pop_tol).err_end
