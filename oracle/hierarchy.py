"""FP64 CPU oracle of the hierarchical time integration (Sec. 4.2) -- TEST INFRASTRUCTURE ONLY.

A step of size dt for a particle set P whose forces a_P (sourced by P alone) are known:
  kick P by a_P dt/2;
  split P into fast particles F (timestep criterion dt_i = sqrt(2 eta eps_i / |a_i|) < dt,
  evaluated on the forces of P) and slow ones S;
  if F is empty: drift P by dt, compute a_P, kick P by a_P dt/2 (a plain kick-drift-kick);
  otherwise: compute a_F (sourced by F alone), kick F by -a_F dt/2; evolve F over dt/2 by the
  same step, recursively; drift S by dt; evolve F over dt/2 again; kick F by -a_F dt/2 with
  the forces F ended with; compute a_P; kick P by a_P dt/2.
This is the operator sequence K_P^P(dt/2) K_F^F(-dt/2) E(H_F, dt/2) D_S(dt) E(H_F, dt/2)
K_F^F(-dt/2) K_P^P(dt/2) of the paper, applied recursively to F.  Every kick uses forces whose
sources and sinks are the same set, so a momentum-conserving force (direct sum, FMM) keeps the
total momentum exactly.  Positions are the uint32 integer coordinates of the force code; a
drift adds rint(v dt 2^32 / L) modulo 2^32 (Sec. 2.10).  Pins: tests/test_oracle_hierarchy.py.
"""
from __future__ import annotations

import numpy as np

TWO32 = 4294967296.0


class State:
    """pos: (3, n) uint32 integer coordinates (unit L / 2^32); vel: (n, 3) float64."""

    def __init__(self, pos_int, vel, mass, L, eps_of):
        self.pos = np.array(pos_int, dtype=np.uint32)
        self.vel = np.array(vel, dtype=np.float64)
        self.mass = np.asarray(mass, np.float64)
        self.L = float(L)
        self.eps = np.asarray(eps_of, np.float64)     # softening length of every particle
        self.n_force = 0                               # particles whose forces were computed


def kick(st: State, idx, acc, dt):
    st.vel[idx] += dt * acc[idx]


def drift(st: State, idx, dt):
    d = np.rint(st.vel[idx] * dt * TWO32 / st.L).astype(np.int64).T
    st.pos[:, idx] = ((st.pos[:, idx].astype(np.int64) + d) % (1 << 32)).astype(np.uint32)


def step(st: State, P, dt, acc_P, force, eta, level=0, max_level=10):
    """Advance the particles P (sorted index array) by dt; acc_P: (n, 3) with the forces of P
    at P; force(idx) -> (n, 3) array with the forces of idx on idx at idx.  Returns the forces
    of P at the end of the step."""
    kick(st, P, acc_P, 0.5 * dt)
    a = np.linalg.norm(acc_P[P], axis=1)
    with np.errstate(divide="ignore"):
        dti = np.sqrt(2.0 * eta * st.eps[P] / a)
    fast = dti < dt if level < max_level else np.zeros(len(P), bool)
    if not fast.any():
        drift(st, P, dt)
        acc = force(P)
        st.n_force += len(P)
        kick(st, P, acc, 0.5 * dt)
        return acc
    F, S = P[fast], P[~fast]
    acc_F = force(F)
    st.n_force += len(F)
    kick(st, F, acc_F, -0.5 * dt)
    acc_F = step(st, F, 0.5 * dt, acc_F, force, eta, level + 1, max_level)
    drift(st, S, dt)
    acc_F = step(st, F, 0.5 * dt, acc_F, force, eta, level + 1, max_level)
    kick(st, F, acc_F, -0.5 * dt)
    acc = force(P)
    st.n_force += len(P)
    kick(st, P, acc, 0.5 * dt)
    return acc
