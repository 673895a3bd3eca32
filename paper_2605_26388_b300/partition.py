"""Element partition and face-trace halo exchange of a Cartesian DGSEM mesh.

The paper's multi-GPU path (Sec. 5, strong and weak scaling) splits the elements into
contiguous ranges and, in every RK stage, exchanges only the face traces on partition faces:
(N+1)^(d-1) n_v values per shared face instead of whole ghost elements, which is all the
Euler residual of an element reads from its neighbours (the Riemann flux at its faces).
This module holds the host logic of that exchange: the partition, the list of shared faces,
packing and unpacking of traces in the state's SoA layout U[v][elem][node] (elements
lexicographic with x fastest, nodes with i fastest), and the exchange itself over
torch.distributed point-to-point messages (gloo on the CPU; the same calls run over NCCL).
"""
from dataclasses import dataclass

import numpy as np


def elem_coords(e: int, nel) -> tuple:
    return (e % nel[0], (e // nel[0]) % nel[1], e // (nel[0] * nel[1]))


def elem_index(c, nel) -> int:
    return c[0] + nel[0] * (c[1] + nel[1] * c[2])


def neighbour(e: int, nel, l: int, side: int) -> int:
    """Periodic neighbour of element e across its face (direction l, side 0 lower / 1 upper)."""
    c = list(elem_coords(e, nel))
    c[l] = (c[l] + (1 if side else -1)) % nel[l]
    return elem_index(c, nel)


def slab_partition(nel, ws: int, axis: int = None) -> list:
    """Contiguous slabs of element layers along `axis` (default: the last axis with more
    than one element): rank r owns layers [r L / ws, (r+1) L / ws).  Returns one sorted array
    of element indices per rank."""
    nel = tuple(nel) + (1,) * (3 - len(nel))
    if axis is None:
        axis = max(l for l in range(3) if nel[l] > 1)
    L = nel[axis]
    if ws > L:
        raise ValueError("more ranks than element layers")
    bounds = [r * L // ws for r in range(ws + 1)]
    n = nel[0] * nel[1] * nel[2]
    layer = np.array([elem_coords(e, nel)[axis] for e in range(n)])
    return [np.nonzero((layer >= bounds[r]) & (layer < bounds[r + 1]))[0] for r in range(ws)]


def face_nodes(N: int, dim: int, l: int, side: int) -> np.ndarray:
    """Node indices of face (l, side) of an element, ordered by the remaining indices
    (lexicographic, lowest direction fastest): the same order on both sides of a face."""
    n1 = N + 1
    nodes = []
    idx = [range(n1) if d < dim else range(1) for d in range(3)]
    fixed = N if side else 0
    for k in idx[2]:
        for j in idx[1]:
            for i in idx[0]:
                ijk = (i, j, k)
                if ijk[l] == fixed:
                    nodes.append(i + n1 * (j + (n1 * k if dim == 3 else 0)))
    return np.array(nodes, dtype=np.int64)


@dataclass
class Halo:
    """One rank's shared faces: for every face this rank owns on a partition boundary, the
    own element, the direction and side, the neighbour element and the rank that owns it."""
    own: np.ndarray
    l: np.ndarray
    side: np.ndarray
    nbr: np.ndarray
    peer: np.ndarray

    def with_peer(self, p: int) -> np.ndarray:
        """Indices of the faces shared with rank p in the canonical order of a face: by
        direction, then by the element on the face's lower side (both ranks of a face compute
        the same key, so their message orders agree)."""
        idx = np.nonzero(self.peer == p)[0]
        low = np.where(self.side[idx] == 1, self.own[idx], self.nbr[idx])
        return idx[np.lexsort((low, self.l[idx]))]


def shared_faces(nel, dim: int, parts: list, rank: int) -> Halo:
    """The faces of rank `rank`'s elements whose neighbour lives on another rank (listed by
    element, direction, side; Halo.with_peer orders them for the messages)."""
    nel3 = tuple(nel) + (1,) * (3 - len(nel))
    owner = np.empty(nel3[0] * nel3[1] * nel3[2], dtype=np.int64)
    for r, p in enumerate(parts):
        owner[p] = r
    own, ls, sides, nbrs, peers = [], [], [], [], []
    for e in parts[rank]:
        for l in range(dim):
            for side in (0, 1):
                en = neighbour(int(e), nel3, l, side)
                if owner[en] != rank:
                    own.append(int(e)); ls.append(l); sides.append(side); nbrs.append(en); peers.append(owner[en])
    a = lambda x: np.array(x, dtype=np.int64)
    return Halo(a(own), a(ls), a(sides), a(nbrs), a(peers))


def pack_traces(U: np.ndarray, halo: Halo, idx: np.ndarray, N: int, dim: int) -> np.ndarray:
    """Own face-node values of the faces halo[idx]: array [len(idx), n_v, (N+1)^(d-1)]."""
    out = []
    for k in idx:
        out.append(U[:, halo.own[k], face_nodes(N, dim, int(halo.l[k]), int(halo.side[k]))])
    nv, nfn = U.shape[0], (N + 1) ** (dim - 1)
    return np.array(out).reshape(len(idx), nv, nfn)


def place_traces(U: np.ndarray, halo: Halo, idx: np.ndarray, traces: np.ndarray, N: int, dim: int) -> None:
    """Write received traces into the neighbour elements' matching face nodes of a local
    state (the neighbour's face on the other side: l, 1 - side)."""
    for t, k in enumerate(idx):
        nodes = face_nodes(N, dim, int(halo.l[k]), 1 - int(halo.side[k]))
        U[:, halo.nbr[k], nodes] = traces[t]


def exchange(U: np.ndarray, halo: Halo, rank: int, ws: int, N: int, dim: int, dist) -> dict:
    """One stage's face-trace exchange: every rank sends each peer the own traces of the
    faces they share and receives the peer's, both in the canonical face order of
    Halo.with_peer; returns {peer: (face indices, received traces)}, trace t belonging to face
    index t of the list (the neighbour's side of that face)."""
    import torch
    received = {}
    reqs, bufs = [], {}
    for p in range(ws):
        if p == rank:
            continue
        idx = halo.with_peer(p)
        if len(idx) == 0:
            continue
        send = torch.from_numpy(np.ascontiguousarray(pack_traces(U, halo, idx, N, dim)))
        recv = torch.empty_like(send)
        bufs[p] = (idx, send, recv)
        reqs.append(dist.isend(send, dst=p))
        reqs.append(dist.irecv(recv, src=p))
    for r in reqs:
        r.wait()
    for p, (idx, _, recv) in bufs.items():
        received[p] = (idx, recv.numpy())
    return received
