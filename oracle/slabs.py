"""Slab decomposition of the oracle step along x, with explicit halo messages
(TEST INFRASTRUCTURE: only tests/ use it).

The lattice is cut into P slabs of whole x planes, one per rank; a rank owns
the populations of its slab and nothing else.  One time step of the method
(R1-R9, see mlb_oracle.c) then needs two exchanges with the two neighbouring
ranks (periodic in x):

1. moment halos.  After the rank's own moments (n^a, j^a, R1), each rank sends
   the H planes next to each face.  H is the reach of the step's force on
   the moments: the acceleration at r reads u* and the pair values on the
   contact shells around r (reach R_s); u* at r' reads the rest force on
   the shells and the attraction region around r' (reach max(R_s, R_a)) and
   the velocities on its shells; every contact value g reads the smoothing
   ball (reach R_b).  So H = R_s + max(R_s, R_a) + R_b.  With the halo the
   rank evaluates R2-R8' on an extended lattice of width w + 2H; values at
   its own planes are those of the whole lattice (the extended lattice's
   wrong periodic wrap is more than H planes away from them).
2. outgoing populations.  After the collision (R9, site-local), the five
   populations of each face site that move across the face (c_x = +1 on the
   right face, -1 on the left one) go to the neighbour, which streams them
   in as if from a ghost plane.  Links that cross a wall (walls normal to y or
   z only) bounce back at their own site, on the rank that owns it.

Every site value is computed by the oracle's own routines from the same
inputs, in the same order, so the decomposed run equals the monolithic
oracle bit for bit.  Two communicators: ranks as threads of one process
(queues) and ranks as processes (torch.distributed point-to-point; gloo on
CPU).
"""
from __future__ import annotations

import dataclasses
import queue
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import Q, accel, attraction_set, collide_local, gfield, moments, shell, velocities

CS2 = 1.0 / 3.0


# ------------------------------------------------------------------ geometry
def halo_depth(lat) -> int:
    """H = R_s + max(R_s, R_a) + R_b (module docstring), plus R_s for every
    further predictor sweep (each reads the partners' u* of the previous one
    on the shells), from the oracle's own enumerated stencils."""
    S = lat.nspecies
    rs = ra = rb = 0
    for a in range(S):
        for b in range(S):
            sab = 0.5 * (lat.sigma[a] + lat.sigma[b])
            d = shell(sab)
            if len(d):
                rs = max(rs, int(np.abs(d).max()))
            if lat.eps[a][b] != 0.0:
                d = attraction_set(sab, lat.lambda_c[a][b])
                if len(d):
                    ra = max(ra, int(np.abs(d).max()))
    for c in range(S):
        rb = max(rb, int(np.floor(lat.kappa * lat.sigma[c] + 1e-12)))
    sweeps = max(1, int(getattr(lat, "predictor_sweeps", 1)))
    extra = (sweeps - 1) * rs if lat.force_scheme != "explicit" else 0
    return rs + max(rs, ra) + rb + extra


def slab_bounds(nx: int, P: int) -> List[Tuple[int, int]]:
    return [(k * nx // P, (k + 1) * nx // P) for k in range(P)]


def _grid(f, lat):
    """[..., N] -> [..., nz, ny, nx] (x fastest)."""
    nx, ny, nz = lat.shape
    return f.reshape(f.shape[:-1] + (nz, ny, nx))


# ------------------------------------------------------------------ communicators
class ThreadComm:
    """P ranks as threads of one process: one FIFO per (source, destination, tag)."""

    def __init__(self, P: int):
        self.P = P
        self._q: Dict[Tuple[int, int, int], queue.Queue] = {}
        self._lock = threading.Lock()

    def _box(self, key):
        with self._lock:
            if key not in self._q:
                self._q[key] = queue.Queue()
            return self._q[key]

    def exchange(self, rank: int, sends: Sequence[Tuple[int, int, np.ndarray]],
                 recvs: Sequence[Tuple[int, int, Tuple[int, ...]]]) -> List[np.ndarray]:
        for dst, tag, arr in sends:
            self._box((rank, dst, tag)).put(np.array(arr, np.float64, copy=True))
        out = []
        for src, tag, shape in recvs:
            a = self._box((src, rank, tag)).get(timeout=120)
            assert a.shape == tuple(shape)
            out.append(a)
        return out


class TorchComm:
    """Ranks as processes: torch.distributed isend / irecv of FP64 tensors."""

    def __init__(self, dist):
        self.dist = dist
        self.P = dist.get_world_size()

    def exchange(self, rank, sends, recvs):
        import torch
        reqs = []
        bufs = []
        for src, tag, shape in recvs:
            t = torch.empty(tuple(shape), dtype=torch.float64)
            bufs.append(t)
            reqs.append(self.dist.irecv(t, src=src, tag=tag))
        keep = []
        for dst, tag, arr in sends:
            t = torch.from_numpy(np.ascontiguousarray(arr, np.float64))
            keep.append(t)
            reqs.append(self.dist.isend(t, dst=dst, tag=tag))
        for r in reqs:
            r.wait()
        return [b.numpy() for b in bufs]


# ------------------------------------------------------------------ one rank
class SlabRank:
    """The state and step of one rank: populations f [S][19][nz][ny][w] of
    the planes x0 .. x1-1 of the lattice `lat`."""

    TAG_MOM_L, TAG_MOM_R, TAG_POP_L, TAG_POP_R = 11, 12, 21, 22

    def __init__(self, lat, rank: int, P: int, f_global: np.ndarray, comm, fext: Optional[np.ndarray] = None,
                 depth: Optional[int] = None):
        if lat.wall_axis == 0:
            raise ValueError("slabs are cut along x: walls normal to x are not supported")
        self.lat, self.rank, self.P, self.comm = lat, rank, P, comm
        nx, ny, nz = lat.shape
        self.x0, self.x1 = slab_bounds(nx, P)[rank]
        self.w = self.x1 - self.x0
        self.H = halo_depth(lat) if depth is None else depth
        if self.w < max(self.H, 1):
            raise ValueError(f"slab of {self.w} planes is thinner than the halo depth {self.H}")
        S = lat.nspecies
        self.f = np.ascontiguousarray(_grid(f_global, lat)[..., self.x0:self.x1])       # [S][Q][nz][ny][w]
        self.lat_w = dataclasses.replace(lat, shape=(self.w, ny, nz))
        self.we = self.w + 2 * self.H
        self.lat_e = dataclasses.replace(lat, shape=(self.we, ny, nz))
        xs = (np.arange(self.x0 - self.H, self.x1 + self.H)) % nx
        self.fext_e = None
        if fext is not None:
            self.fext_e = np.ascontiguousarray(_grid(np.asarray(fext, np.float64), lat)[..., xs]).reshape(S, 3, -1)
        X, Y, Z = np.meshgrid(np.arange(self.H, self.H + self.w), np.arange(ny), np.arange(nz), indexing="ij")
        self.owned = np.ascontiguousarray((X + self.we * (Y + ny * Z)).transpose(2, 1, 0).reshape(-1), np.int64)
        self.left, self.right = (rank - 1) % P, (rank + 1) % P
        c, wts = velocities()
        self.c, self.wts = c.astype(int), wts
        self.opp = np.array([int(np.where((c == -c[i]).all(1))[0][0]) for i in range(Q)])

    # R1 and the moment halo
    def _moments_extended(self):
        lat, S, H, w = self.lat, self.lat.nspecies, self.H, self.w
        nx, ny, nz = lat.shape
        n, j = moments(self.lat_w, self.f.reshape(S, Q, -1))
        m = np.concatenate([n.reshape(S, nz, ny, w), j.reshape(3 * S, nz, ny, w)], 0)   # [4S][nz][ny][w]
        shape = (4 * S, nz, ny, H)
        from_left, from_right = self.comm.exchange(
            self.rank,
            [(self.left, self.TAG_MOM_L, m[..., :H]), (self.right, self.TAG_MOM_R, m[..., w - H:])],
            [(self.left, self.TAG_MOM_R, shape), (self.right, self.TAG_MOM_L, shape)])
        me = np.concatenate([from_left, m, from_right], -1)
        n_e = np.ascontiguousarray(me[:S]).reshape(S, -1)
        j_e = np.ascontiguousarray(me[S:]).reshape(S, 3, -1)
        return n, j, n_e, j_e

    def step(self):
        lat, S, w = self.lat, self.lat.nspecies, self.w
        nx, ny, nz = lat.shape
        n, j, n_e, j_e = self._moments_extended()
        # R2-R8' on the extended lattice, at the rank's own sites
        g_e, _, _ = gfield(self.lat_e, n_e)
        acc = accel(self.lat_e, n_e, j_e, g_e, self.fext_e, sites=self.owned)            # [S][3][M]
        # R9: site-local collision
        M = w * ny * nz
        fpost = collide_local(lat, self.f.reshape(S, Q, M).transpose(2, 0, 1), n.T, j.transpose(2, 0, 1),
                              acc.transpose(2, 0, 1))                                    # [M][S][Q]
        fp = np.ascontiguousarray(fpost.transpose(1, 2, 0)).reshape(S, Q, nz, ny, w)
        # outgoing faces: populations with c_x = +1 leave through the right face, -1 through the left
        right_i = [i for i in range(Q) if self.c[i][0] == 1]
        left_i = [i for i in range(Q) if self.c[i][0] == -1]
        shp = (S, len(right_i), nz, ny)
        to_right = np.stack([fp[:, i, :, :, w - 1] for i in right_i], 1)
        to_left = np.stack([fp[:, i, :, :, 0] for i in left_i], 1)
        from_left, from_right = self.comm.exchange(
            self.rank, [(self.right, self.TAG_POP_R, to_right), (self.left, self.TAG_POP_L, to_left)],
            [(self.left, self.TAG_POP_R, shp), (self.right, self.TAG_POP_L, shp)])
        # stream from the planes -1 .. w (ghosts at both ends) into the rank's planes
        ext = np.zeros((S, Q, nz, ny, w + 2))
        ext[..., 1:w + 1] = fp
        for k, i in enumerate(right_i):
            ext[:, i, :, :, 0] = from_left[:, k]
        for k, i in enumerate(left_i):
            ext[:, i, :, :, w + 1] = from_right[:, k]
        self.f = self._stream(ext, n.reshape(S, nz, ny, w))

    def _stream(self, ext, n_own):
        lat, S, w = self.lat, self.lat.nspecies, self.w
        nx, ny, nz = lat.shape
        out = np.full((S, Q, nz, ny, w), np.nan)
        Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(w + 2), indexing="ij")   # X: extended plane
        for i in range(Q):
            cx, cy, cz = (int(v) for v in self.c[i])
            ty, tz, tx = Y + cy, Z + cz, X + cx
            cross = np.zeros(X.shape, bool)
            if lat.wall_axis == 1:
                cross |= (ty < 0) | (ty >= ny)
            else:
                ty %= ny
            if lat.wall_axis == 2:
                cross |= (tz < 0) | (tz >= nz)
            else:
                tz %= nz
            own_src = (X >= 1) & (X <= w)
            move = ~cross & (tx >= 1) & (tx <= w)
            out[:, i, tz[move], ty[move], tx[move] - 1] = ext[:, i, Z[move], Y[move], X[move]]
            bb = cross & own_src
            if bb.any():
                # halfway bounce-back on a moving wall, as the monolithic oracle computes it
                ax = lat.wall_axis
                coord = (Y if ax == 1 else Z)[bb]
                cax = cy if ax == 1 else cz
                lo = coord + cax < 0
                for side, uw in ((lo, lat.wall_u_lo), (~lo, lat.wall_u_hi)):
                    if not side.any():
                        continue
                    cuw = float(self.c[i][0]) * uw[0] + float(self.c[i][1]) * uw[1] + float(self.c[i][2]) * uw[2]
                    zz, yy, xx = Z[bb][side], Y[bb][side], X[bb][side]
                    src = ext[:, i, zz, yy, xx]
                    na = n_own[:, zz, yy, xx - 1]
                    out[:, self.opp[i], zz, yy, xx - 1] = src - 2.0 * self.wts[i] * na * cuw / CS2
        assert not np.isnan(out).any()
        return out


# ------------------------------------------------------------------ drivers
def run_threads(lat, f: np.ndarray, nsteps: int, P: int, fext=None, depth: Optional[int] = None) -> np.ndarray:
    """Advance the [S][19][N] populations by nsteps with P ranks as threads;
    returns the gathered populations (f is not modified)."""
    comm = ThreadComm(P)
    ranks = [SlabRank(lat, r, P, f, comm, fext, depth) for r in range(P)]
    errors: List[BaseException] = []

    def work(rk):
        try:
            for _ in range(nsteps):
                rk.step()
        except BaseException as e:   # surfaced below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(rk,)) for rk in ranks]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return gather(lat, [rk.f for rk in ranks])


def gather(lat, slabs: Sequence[np.ndarray]) -> np.ndarray:
    S = lat.nspecies
    return np.ascontiguousarray(np.concatenate(slabs, -1)).reshape(S, Q, -1)
