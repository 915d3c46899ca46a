"""Spatial decomposition of the DPD-CGMD system into x-slabs, one per rank.

The channel's long axis x is periodic; each of R ranks owns the slab
[r Lx/R, (r + 1) Lx/R).  The step needs, per force evaluation:

* ownership: plasma and wall particles by their own x; a platelet as a
  whole by the x of its centre of mass (its bonded terms -- bonds of Eq. 2,
  angles -- then never span ranks);
* a ghost exchange: every rank sends the state of the particles it owns
  that lie within pair reach of another rank's owned region (the x-extent
  of its owned particles: platelets reach beyond their slab) -- reach 1.0 for
  plasma and wall particles (the DPD cut-off of Eq. 1 and 3), 5.0 for
  platelet particles (the receptor Morse cut-off of Eq. 4);
* half-shell pairs: a pair is evaluated once, by the rank that owns its
  particle of lower id; the force on a ghost partner is sent back to the
  partner's owner (the reverse-force exchange) and added there;
* migration at a rebuild: particles whose owner changed move with their
  state;
* FP64 reductions (kinetic energy, momentum, ...) summed over the ranks.

Pairs and bonded terms are evaluated by callables handed in, so the same
logic serves any force evaluator; the counter-based pair noise (keyed on the
two ids and the time index) gives a pair the same random force whichever
rank evaluates it.  Communication goes through torch.distributed
point-to-point messages (NCCL send/recv between devices, each into the
receiving device's own memory; gloo on host ranks).
"""
from __future__ import annotations

import numpy as np

REACH_FLUID = 1.0     # DPD cut-off (Eq. 1, Eq. 3)
REACH_PLT = 5.0       # receptor Morse cut-off (Eq. 4), the longest platelet pair reach

FIELDS = ("id", "x", "v", "tag", "X0")


def _dist():
    import torch.distributed as dist
    return dist


class Slabs:
    """Slab geometry and ownership rules for `world` ranks over a box."""

    def __init__(self, box, rank, world):
        self.L = np.asarray(box, dtype=np.float64)
        self.rank, self.world = int(rank), int(world)
        self.w = self.L[0] / self.world

    def slab_of(self, x0):
        """Rank whose slab holds coordinate x0 (periodic in x)."""
        return np.minimum((np.mod(x0, self.L[0]) // self.w).astype(np.int64), self.world - 1)

    def owners(self, x, tag):
        """Owner rank of each particle: by its x, platelet members by the x of
        their platelet's centre of mass (minimum image about a member)."""
        own = self.slab_of(x[:, 0])
        plt = tag >= 0
        if plt.any():
            pid = (tag[plt] & ~(1 << 30)).astype(np.int64)
            xp = x[plt, 0]
            P = int(pid.max()) + 1
            ref = np.zeros(P)
            ref[pid] = xp                       # any member as the image reference
            d = xp - ref[pid]
            d -= self.L[0] * np.round(d / self.L[0])
            cnt = np.bincount(pid, minlength=P)
            com = ref + np.bincount(pid, weights=d, minlength=P) / np.maximum(cnt, 1)
            own[plt] = self.slab_of(com[pid])
        return own

    def region(self, x):
        """x-interval of the owned positions x (unwrapped about the slab
        centre): (centre, lo offset, hi offset)."""
        c = (self.rank + 0.5) * self.w
        if len(x) == 0:
            return c, -0.5 * self.w, 0.5 * self.w
        d = x[:, 0] - c
        d -= self.L[0] * np.round(d / self.L[0])
        return c, min(float(d.min()), -0.5 * self.w), max(float(d.max()), 0.5 * self.w)

    def within(self, x0, reach, region):
        """Positions x0 within `reach` (per particle) of an owned region."""
        c, lo, hi = region
        d = x0 - c
        d -= self.L[0] * np.round(d / self.L[0])
        return (d >= lo - reach) & (d <= hi + reach)


def exchange(payloads, world, rank, tag=0):
    """Send payloads[q] (a dict of arrays, or None) to every rank q != rank and
    return what every other rank sent here: {q: dict}.  Sizes go first, then
    the arrays, as point-to-point messages (non-blocking, so no ordering
    deadlock)."""
    import torch
    dist = _dist()
    out = {}
    # sizes
    sends, recvs, sizes = [], [], {}
    for q in range(world):
        if q == rank:
            continue
        p = payloads.get(q)
        n = 0 if p is None else len(p["id"])
        sends.append(dist.isend(torch.tensor([n], dtype=torch.int64), q, tag=tag))
        sizes[q] = torch.zeros(1, dtype=torch.int64)
        recvs.append(dist.irecv(sizes[q], q, tag=tag))
    for h in sends + recvs:
        h.wait()
    # arrays, packed as one float64 block and one int64 block per peer
    sends, recvs, bufs = [], [], {}
    for q in range(world):
        if q == rank:
            continue
        p = payloads.get(q)
        if p is not None and len(p["id"]):
            fl = np.concatenate([np.asarray(p[k], np.float64).reshape(len(p["id"]), -1) for k in p.get("_f", ())],
                                axis=1) if p.get("_f") else np.zeros((len(p["id"]), 0))
            it = np.stack([np.asarray(p[k], np.int64) for k in p.get("_i", ())], axis=1)
            sends.append(dist.isend(torch.from_numpy(np.ascontiguousarray(fl)), q, tag=tag + 1))
            sends.append(dist.isend(torch.from_numpy(np.ascontiguousarray(it)), q, tag=tag + 2))
        m = int(sizes[q].item())
        if m:
            bufs[q] = (torch.zeros((m, payloads["_fw"]), dtype=torch.float64),
                       torch.zeros((m, payloads["_iw"]), dtype=torch.int64))
            recvs.append(dist.irecv(bufs[q][0], q, tag=tag + 1))
            recvs.append(dist.irecv(bufs[q][1], q, tag=tag + 2))
    for h in sends + recvs:
        h.wait()
    for q, (fl, it) in bufs.items():
        out[q] = (fl.numpy(), it.numpy())
    return out


class SlabSystem:
    """The particles one rank owns, with the exchanges of a force
    evaluation.  State arrays are in the rank's own order; `id` maps them to
    global particle ids."""

    def __init__(self, slabs, id, x, v, tag, X0):
        self.s = slabs
        self.id = np.asarray(id, np.int64)
        self.x = np.asarray(x, np.float64)
        self.v = np.asarray(v, np.float64)
        self.tag = np.asarray(tag, np.int64)
        self.X0 = np.asarray(X0, np.float64)

    @classmethod
    def scatter(cls, slabs, x, v, tag, X0):
        """This rank's share of a whole system known on every rank (set-up)."""
        own = slabs.owners(x, np.asarray(tag))
        m = own == slabs.rank
        return cls(slabs, np.nonzero(m)[0], x[m], v[m], np.asarray(tag)[m], X0[m])

    def _pack(self, sel):
        return {"id": self.id[sel], "x": self.x[sel], "v": self.v[sel], "X0": self.X0[sel], "tag": self.tag[sel],
                "_f": ("x", "v", "X0"), "_i": ("id", "tag")}

    @staticmethod
    def _unpack(fl, it):
        return dict(x=fl[:, 0:3], v=fl[:, 3:6], X0=fl[:, 6:9], id=it[:, 0], tag=it[:, 1])

    def regions(self):
        """Every rank's owned region (all-gathered)."""
        import torch
        dist = _dist()
        c, lo, hi = self.s.region(self.x)
        t = torch.tensor([c, lo, hi], dtype=torch.float64)
        allr = [torch.zeros(3, dtype=torch.float64) for _ in range(self.s.world)]
        dist.all_gather(allr, t)
        return [tuple(a.tolist()) for a in allr]

    def ghosts(self):
        """Ghost exchange: the state of every other rank's particles within
        pair reach of this rank's owned region.  Returns a dict of arrays."""
        regs = self.regions()
        reach = np.where(self.tag >= 0, REACH_PLT, REACH_FLUID)
        pay = {"_fw": 9, "_iw": 2}
        for q in range(self.s.world):
            if q == self.s.rank:
                continue
            sel = self.s.within(self.x[:, 0], reach, regs[q])
            pay[q] = self._pack(sel) if sel.any() else None
        got = exchange(pay, self.s.world, self.s.rank, tag=10)
        parts = []
        for q, (fl, it) in got.items():
            d = self._unpack(fl, it)
            d["src"] = np.full(len(d["id"]), q, np.int64)      # the ghost's owner
            parts.append(d)
        if not parts:
            return dict(x=np.zeros((0, 3)), v=np.zeros((0, 3)), X0=np.zeros((0, 3)), id=np.zeros(0, np.int64),
                        tag=np.zeros(0, np.int64), src=np.zeros(0, np.int64))
        return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}

    def forces(self, pair_force, bonded_force, reach_pair, body_force=0.0):
        """Forces on the owned particles.

        pair_force(x, v, tag, id, X0, pairs) -> F[npair, 3]: force on pairs[:, 0]
        from pairs[:, 1] over the local arrays (owned then ghosts).
        bonded_force(id, x) -> f[n_owned, 3]: the bonded terms of the owned
        platelets (all of whose members are owned here).
        reach_pair(tag_a, tag_b) -> the pair reach for those particle kinds."""
        g = self.ghosts()
        n = len(self.id)
        loc = {k: np.concatenate([getattr(self, k), g[k]]) for k in ("id", "x", "v", "tag", "X0")}
        # half-shell pairs evaluated here: the lower-id particle is owned
        a, b = self._pairs(loc, n, reach_pair)
        F = pair_force(loc["x"], loc["v"], loc["tag"], loc["id"], loc["X0"], np.stack([a, b], 1)) if len(a) else \
            np.zeros((0, 3))
        f = np.zeros((len(loc["id"]), 3))
        np.add.at(f, a, F)
        np.add.at(f, b, -F)
        # reverse forces: the ghosts' shares go back to their owners (the
        # ranks they came from)
        fg = f[n:]
        nz = np.abs(fg).sum(1) > 0
        pay = {"_fw": 3, "_iw": 1}
        src = g["src"]
        for q in range(self.s.world):
            if q == self.s.rank:
                continue
            sel = nz & (src == q)
            pay[q] = {"id": g["id"][sel], "f": fg[sel], "_f": ("f",), "_i": ("id",)} if sel.any() else None
        back = exchange(pay, self.s.world, self.s.rank, tag=20)
        fo = f[:n].copy()
        pos = {int(i): k for k, i in enumerate(self.id)}
        for fl, it in back.values():
            for row, gid in zip(fl, it[:, 0]):
                fo[pos[int(gid)]] += row
        fo += bonded_force(self.id, self.x)
        fo[self.tag != -2, 0] += body_force
        return fo

    def _pairs(self, loc, n, reach_pair):
        """Pairs (a owned, b local) with id_a < id_b within reach (brute force
        over the local set; a device build would use the cell lists)."""
        x, tag, ids = loc["x"], loc["tag"], loc["id"]
        L = self.s.L
        A, B = [], []
        for a0 in range(0, n, 2048):
            a1 = min(n, a0 + 2048)
            d = x[a0:a1, None, :] - x[None, :, :]
            d[..., 0] -= L[0] * np.round(d[..., 0] / L[0])
            d[..., 2] -= L[2] * np.round(d[..., 2] / L[2])
            r2 = (d * d).sum(-1)
            ta, tb = tag[a0:a1, None], tag[None, :]
            reach = reach_pair(ta, tb)
            ok = (r2 < reach * reach) & (ids[a0:a1, None] < ids[None, :])
            ia, ib = np.nonzero(ok)
            A.append(ia + a0)
            B.append(ib)
        return np.concatenate(A), np.concatenate(B)

    def migrate(self):
        """Ownership after the particles moved: every particle whose owner
        changed goes, with its state, to the new owner (at a list rebuild)."""
        # whole-platelet centres need every member; members are all owned here
        own = self.s.owners(self.x, self.tag)
        pay = {"_fw": 9, "_iw": 2}
        for q in range(self.s.world):
            if q != self.s.rank:
                sel = own == q
                pay[q] = self._pack(sel) if sel.any() else None
        got = exchange(pay, self.s.world, self.s.rank, tag=30)
        keep = own == self.s.rank
        parts = [dict(id=self.id[keep], x=self.x[keep], v=self.v[keep], X0=self.X0[keep], tag=self.tag[keep])]
        parts += [self._unpack(fl, it) for fl, it in got.values()]
        for k in ("id", "x", "v", "X0", "tag"):
            setattr(self, k, np.concatenate([p[k] for p in parts]))
        order = np.argsort(self.id, kind="stable")
        for k in ("id", "x", "v", "X0", "tag"):
            setattr(self, k, getattr(self, k)[order])

    def reduce_fp64(self, values):
        """Sum of per-rank FP64 values over every rank."""
        import torch
        dist = _dist()
        t = torch.tensor(np.asarray(values, np.float64), dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()
