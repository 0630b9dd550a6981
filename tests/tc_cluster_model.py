"""Model of the synchronisation protocol of the clustered tcgen05 H_eff psi
kernel (paper_2503_20700_gb300/csrc/hpsi_tc.cu), run on the CPU over plans
made by the real planner (tests/cpp/tc_plan_dump.cpp).

Every CTA of a cluster has three roles, written here as coroutines that
yield the barrier phase they wait for: the producer (stage fills), the MMA
issuer (stage 1 of this CTA's super-chunks, stage 2 of every piece, one
count per piece on every CTA's piece-read barrier, drain signals) and the
converters (the in-order wait on the piece-read barrier and its
acknowledgement, conversion of this CTA's pieces into the buffers of its
group, drains).  Barriers complete a phase after `count` arrivals and are
probed by parity, like mbarriers.  MMA and copy completions are queued and
retired in a random order against the roles, which are also scheduled at
random.  The model reports a deadlock (no role can proceed) and checks
hazards: a piece buffer written while its previous piece is unread, an MMA
reading a buffer that does not hold its piece, X' overwritten before its
pieces are converted, a stage refilled while read.

The walk and the issue order of stage 1 follow the kernel's Walk, walk_*,
s1_now and s1_issued; a change to either side must be made to both."""
from __future__ import annotations

import random
from collections import deque

W1, PW, NSTAGE, NXB = 256, 32, 3, 2


class Hazard(Exception):
    pass


def parse_plan(text):
    lines = iter(text.splitlines())
    check = next(lines).split(None, 1)[1]
    cluster = int(next(lines).split()[1])
    tile_n = int(next(lines).split()[1])
    nb = int(next(lines).split()[1])
    blocks = [tuple(map(int, next(lines).split())) for _ in range(nb)]
    ni = int(next(lines).split()[1])
    items = [tuple(map(int, next(lines).split())) for _ in range(ni)]
    nt = int(next(lines).split()[1])
    tasks = [tuple(map(int, next(lines).split())) for _ in range(nt)]
    nc = int(next(lines).split()[1])
    lists = []
    for _ in range(nc):
        f = next(lines).split()
        lists.append([tuple(map(int, e.split(","))) for e in f[1:]])
    return dict(check=check, cluster=cluster, tile_n=tile_n, blocks=blocks, items=items, tasks=tasks,
                lists=lists)


class Barrier:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, 0, 0

    def arrive(self):
        self.pending += 1
        if self.pending == self.count:
            self.pending, self.phase = 0, self.phase + 1

    def done(self, parity):
        # the phase with this parity is complete when the current one has the other parity
        return (self.phase & 1) != parity


class Walk:
    """The piece sequence of one CTA (kernel: struct Walk and walk_*)."""

    def __init__(self, plan, lst, rank, drain_terms):
        self.plan, self.list, self.rank, self.drain_terms = plan, lst, rank, drain_terms
        self.t = 0
        self.valid = len(lst) > 0
        if self.valid:
            self._task()

    def _task(self):
        self.sl = self.list[self.t]
        self.tk = self.plan["tasks"][self.sl[0]]
        m, n = self.plan["blocks"][self.tk[0]]
        self.N = (min(self.plan["tile_n"], n - self.tk[2]) + 15) & ~15
        self.ii, self.k, self.jc, self.p, self.sct = self.tk[3], 0, 0, 0, 0
        self.it = self.plan["items"][self.ii]
        self.acc = self.it[1]

    def copy(self):
        c = Walk.__new__(Walk)
        c.__dict__.update(self.__dict__)
        return c

    def ghost(self):
        return self.sl[3] != 0

    def owned(self):
        return not self.sl[3] and self.sct % self.sl[2] == self.rank - self.sl[1]

    def sc_width(self):
        return min(W1, self.it[1] - self.jc)

    def sc_pieces(self):
        return (self.sc_width() + PW - 1) // PW

    def last_piece(self):
        return self.p + 1 >= self.sc_pieces()

    def drain_point(self):
        last_of_item = self.last_piece() and self.jc + W1 >= self.it[1]
        return last_of_item and (self.acc >= self.drain_terms or self.k + 1 == self.tk[4])

    def next(self):
        drained = self.drain_point()
        if not self.last_piece():
            self.p += 1
            return
        self.p = 0
        self.sct += 1
        self.jc += W1
        if self.jc < self.it[1]:
            return
        self.jc, self.p = 0, 0
        self.ii += 1
        self.k += 1
        if self.k < self.tk[4]:
            self.it = self.plan["items"][self.ii]
            self.acc = self.it[1] if drained else self.acc + self.it[1]
            return
        self.t += 1
        if self.t >= len(self.list):
            self.valid = False
            return
        self._task()

    def next_sc(self):
        self.p = self.sc_pieces() - 1
        self.next()

    def next_owned(self):
        self.next_sc()
        while self.valid and not self.owned():
            self.next_sc()

    def first_owned(self):
        if self.valid and not self.owned():
            self.next_owned()

    def s1_blocks(self):
        return (self.it[0] + 15) >> 4

    def s2_kblocks(self):
        return min(2, (self.it[1] - self.jc - PW * self.p + 15) >> 4)

    def same_sc(self, o):
        return self.t == o.t and self.sct == o.sct


class S1Order:
    """Issue order of stage 1 (kernel: S1Order, s1_now, s1_issued)."""

    def __init__(self, s2w):
        self.w = s2w.copy()
        self.w.first_owned()
        self.done = 0
        self.held = None

    def now(self, s2w):
        if self.held == (s2w.t, s2w.sct) and s2w.last_piece():
            self.held = None
        if self.held is not None or not self.w.valid:
            return 0
        nb = self.w.s1_blocks()
        if self.w.same_sc(s2w):
            return nb - self.done
        if s2w.owned():
            if not s2w.last_piece():
                return 0
            n = s2w.copy()
            n.next_sc()
            return nb - self.done if (n.valid and n.same_sc(self.w)) else 0
        np_ = s2w.sc_pieces()
        return max(0, (nb * (s2w.p + 1) + np_ - 1) // np_ - self.done)

    def issued(self, s2w, k):
        self.done += k
        if self.done < self.w.s1_blocks():
            return
        self.held = (self.w.t, self.w.sct)
        if self.w.same_sc(s2w) and s2w.last_piece():
            self.held = None
        self.w.next_owned()
        self.done = 0


class CTA:
    def __init__(self, C):
        self.FULL = [Barrier(1) for _ in range(NSTAGE)]
        self.EMPTY = [Barrier(1) for _ in range(NSTAGE)]
        self.XPF, self.XPE = Barrier(1), Barrier(1)
        self.XF = [Barrier(1) for _ in range(NXB)]
        self.XE = [Barrier(C) for _ in range(NXB)]
        self.XA = [Barrier(1) for _ in range(NXB)]
        self.SF, self.SE = Barrier(1), Barrier(1)
        self.mq, self.tq = deque(), deque()  # MMA completions, copy completions
        self.buf = [dict(content=None, consumed=True, reading=False) for _ in range(NXB)]
        self.xp = dict(sc=None, left=0)
        self.stage = [dict(filled=None, reading=False) for _ in range(NSTAGE)]


def run_cluster(plan, k, seed=0, drain_terms=1024, ack=True):
    """One cluster of the plan under a random schedule: ("ok", steps),
    ("deadlock", [(role, wait), ...]) or ("hazard", message).  ack=False
    removes the converters' in-order wait and acknowledgement (a protocol
    the kernel must not use), for checking that the model finds its faults."""
    C = plan["cluster"]
    rng = random.Random(seed)
    lists = plan["lists"][k * C:(k + 1) * C]
    cl = [CTA(C) for _ in range(C)]

    def producer(j):
        me, q = cl[j], [0]

        def fill():
            s = q[0] % NSTAGE
            yield ("producer EMPTY", me.EMPTY[s], ((q[0] // NSTAGE) & 1) ^ 1)
            if me.stage[s]["reading"]:
                raise Hazard("cta %d: stage %d refilled while read" % (j, s))
            n = q[0]
            me.tq.append(lambda: (me.stage[s].update(filled=n), me.FULL[s].arrive()))
            q[0] += 1

        s2w = Walk(plan, lists[j], j, drain_terms)
        o = S1Order(s2w)
        while s2w.valid:
            kk = o.now(s2w)
            for _ in range(kk):
                yield from fill()
            if kk:
                o.issued(s2w, kk)
            if not s2w.ghost():
                for _ in range(s2w.s2_kblocks()):
                    yield from fill()
            s2w.next()

    def mma(j):
        me = cl[j]
        st = dict(q=0, nd=0, nsc=0, g=0, need_se=False)
        xfu = [0] * NXB

        def take():
            s = st["q"] % NSTAGE
            yield ("mma FULL", me.FULL[s], (st["q"] // NSTAGE) & 1)
            if me.stage[s]["filled"] != st["q"]:
                raise Hazard("cta %d: stage %d not filled" % (j, s))
            me.stage[s]["reading"] = True
            me.mq.append(lambda: (me.stage[s].update(reading=False), me.EMPTY[s].arrive()))
            st["q"] += 1

        def stage1(w, k0, k1):
            if k0 == 0:
                if st["nsc"] >= 1:
                    yield ("mma XPE", me.XPE, (st["nsc"] - 1) & 1)
                if me.xp["left"] != 0:
                    raise Hazard("cta %d: X' overwritten before its pieces were read" % j)
            for _ in range(k0, k1):
                yield from take()
            if k1 == w.s1_blocks():
                sc, npc = (w.t, w.sct), w.sc_pieces()
                me.mq.append(lambda: (me.xp.update(sc=sc, left=npc), me.XPF.arrive()))
                st["nsc"] += 1

        def stage2(w):
            g = st["g"]
            b = g % NXB
            if ack:
                yield ("mma XA g=%d" % g, me.XA[b], (g // NXB) & 1)
            yield ("mma XF g=%d" % g, me.XF[b], xfu[b] & 1)
            xfu[b] += 1
            bf = me.buf[b]
            if bf["content"] != g:
                raise Hazard("cta %d piece %d: buffer %d holds piece %s" % (j, g, b, bf["content"]))
            bf["reading"] = True
            if st["need_se"]:
                yield ("mma SE", me.SE, (st["nd"] - 1) & 1)
                st["need_se"] = False
            for _ in range(w.s2_kblocks()):
                yield from take()

            def read_done():
                bf["reading"] = False
                bf["consumed"] = True
                for c in cl:
                    c.XE[b].arrive()
            me.mq.append(read_done)
            st["g"] += 1
            if w.drain_point():
                me.mq.append(lambda: me.SF.arrive())
                st["nd"] += 1
                st["need_se"] = True

        def ghost_piece():
            g = st["g"]
            b = g % NXB
            if ack:
                yield ("ghost XA g=%d" % g, me.XA[b], (g // NXB) & 1)
            elif g >= NXB:
                yield ("ghost XE g=%d" % g, me.XE[b], ((g // NXB) - 1) & 1)
            me.mq.append(lambda: [c.XE[b].arrive() for c in cl])
            st["g"] += 1

        s2w = Walk(plan, lists[j], j, drain_terms)
        o = S1Order(s2w)
        while s2w.valid:
            kk = o.now(s2w)
            if kk:
                yield from stage1(o.w, o.done, o.done + kk)
                o.issued(s2w, kk)
            if s2w.ghost():
                yield from ghost_piece()
            else:
                yield from stage2(s2w)
            s2w.next()

    def converters(j):
        me = cl[j]
        st = dict(nd=0, nsc=0, g=0)

        def convert(w):
            g = st["g"]
            b = g % NXB
            if not ack and g >= NXB:
                yield ("converters XE g=%d" % g, me.XE[b], ((g // NXB) - 1) & 1)
            if w.p == 0:
                yield ("converters XPF", me.XPF, st["nsc"] & 1)
            if me.xp["sc"] != (w.t, w.sct):
                raise Hazard("cta %d: X' holds %s, piece of %s" % (j, me.xp["sc"], (w.t, w.sct)))
            me.xp["left"] -= 1
            if w.last_piece():
                me.XPE.arrive()
                st["nsc"] += 1
            g0, gn = w.sl[1], w.sl[2]
            for m in range(g0, g0 + gn):
                bf = cl[m].buf[b]
                if bf["reading"] or not bf["consumed"]:
                    raise Hazard("piece %d written into cta %d buffer %d holding unread piece %s"
                                 % (g, m, b, bf["content"]))
            # this CTA's copy at once, the peer's by the copy engine
            me.buf[b].update(content=g, consumed=False)
            me.XF[b].arrive()
            for m in range(g0, g0 + gn):
                if m != j:
                    peer = cl[m]

                    def land(peer=peer, b=b, g=g):
                        peer.buf[b].update(content=g, consumed=False)
                        peer.XF[b].arrive()
                    me.tq.append(land)

        def drain():
            yield ("converters SF", me.SF, st["nd"] & 1)
            me.SE.arrive()
            st["nd"] += 1

        w = Walk(plan, lists[j], j, drain_terms)
        pend = False
        while w.valid:
            g = st["g"]
            if ack:
                if g >= NXB:
                    yield ("converters XE g=%d" % g, me.XE[g % NXB], ((g // NXB) - 1) & 1)
                me.XA[g % NXB].arrive()
            if w.owned():
                yield from convert(w)
            if pend:
                yield from drain()
            pend = (not w.ghost()) and w.drain_point()
            st["g"] += 1
            w.next()
        if pend:
            yield from drain()

    roles = []
    for j in range(C):
        for name, f in (("producer", producer), ("mma", mma), ("converters", converters)):
            roles.append(["%s%d" % (name, j), f(j), None])
    live = list(roles)
    steps = 0
    while True:
        queues = [c.mq for c in cl if c.mq] + [c.tq for c in cl if c.tq]
        ready = [r for r in live if r[2] is None or r[2][1].done(r[2][2])]
        cands = [("role", r) for r in ready] + [("queue", q) for q in queues]
        if not cands:
            if live:
                return "deadlock", [(r[0], r[2][0]) for r in live]
            return "ok", steps
        kind, x = rng.choice(cands)
        steps += 1
        try:
            if kind == "queue":
                x.popleft()()
            else:
                try:
                    x[2] = next(x[1])
                except StopIteration:
                    live.remove(x)
        except Hazard as e:
            return "hazard", str(e)
