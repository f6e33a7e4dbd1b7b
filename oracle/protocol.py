"""Sequential simulator of the LightKernel host<->GPU dispatch protocol.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The model follows Burgio, "Enabling predictable parallelism in single-GPU
systems with persistent CUDA threads":

* Sec. II.C: one persistent block per SM, pinned at boot; work is handed to a
  chosen cluster of SMs.  A cluster here is a set of pinned blocks (ranks);
  rank 0 is the cluster's master.
* Sec. II.D and Table 1: each cluster has two integer mailboxes.  ``to_GPU``
  carries THREAD_NOP=4, THREAD_EXIT=8 or THREAD_WORK=16+op from the host;
  ``from_GPU`` carries THREAD_INIT=0, THREAD_FINISHED=1, THREAD_WORKING=2 or
  THREAD_NOP=4 from the master thread.

Two protocol variants are simulated, both as interleavings of atomic steps of
independent agents (host producers, a disposer that posts EXIT, one master
and the other ranks of every cluster):

``mailbox``  the paper's one-deep dual mailbox.  The host may post when the
             mailbox is idle (from_GPU in {INIT, NOP}, to_GPU = NOP); the
             master answers WORKING, relays the descriptor to the other ranks,
             and once every rank has arrived writes FINISHED; the host's wait
             sees FINISHED and re-arms with to_GPU = NOP; the master
             acknowledges with from_GPU = NOP.  (The paper lists NOP in both
             directions without giving the handshake; this four-phase reading
             is the one used throughout.)
``ring``     the multi-slot generalisation: per cluster a ring of R slots, each
             published with a monotone sequence number; producers take tickets
             (ticket order = FIFO order), the master takes slot ``head`` when
             its sequence number is ``head + 1``, relays it through a D-deep
             broadcast ring, and the last rank to arrive publishes
             ``done = seq``.

Each rank appends (seq, op, smid) to its own log when it runs its share.  The
logs are what the execution-log checker (``oracle.check_exec_log``) reads, for
simulated runs and for the GPU's own log alike.  Completion soundness (no
completion before every share of the descriptor has run) and slot reuse (no
slot rewritten before its master took it) are checked at the step where they
could break.

``mutate`` plants a single mistake in the simulated protocol; tests use it to
show the checker catches each class of error.
"""
from __future__ import annotations

import random
from dataclasses import dataclass

# Table 1 (Sec. II.D)
FROM_GPU = {"THREAD_INIT": 0, "THREAD_FINISHED": 1, "THREAD_WORKING": 2, "THREAD_NOP": 4}
TO_GPU = {"THREAD_NOP": 4, "THREAD_EXIT": 8, "THREAD_WORK": 16}
INIT, FINISHED, WORKING, F_NOP = 0, 1, 2, 4
T_NOP, T_EXIT, T_WORK = 4, 8, 16
EXIT_OP = -1

MUTATIONS = ("skip_share", "double_share", "wrong_smid", "early_complete",
             "ignore_bcast_free", "ignore_ring_full", "wrong_op")


@dataclass
class Instance:
    sizes: tuple            # ranks per cluster
    smids: tuple            # smids[c][r]: SM that rank r of cluster c is pinned to
    jobs: tuple             # jobs[p]: tuple of (cluster, op) posted by producer p, in order
    mode: str = "ring"      # "ring" or "mailbox"
    ring_depth: int = 2
    bcast_depth: int = 1
    mutate: str | None = None


class State:
    """Whole-system state; plain lists so that a copy is cheap."""

    def __init__(self, inst: Instance):
        C = len(inst.sizes)
        self.inst = inst
        # host-visible words
        self.ring = [[(0, 0)] * inst.ring_depth for _ in range(C)]   # (seq, op)
        self.tail = [0] * C
        self.done = [0] * C
        self.to_gpu = [T_NOP] * C
        self.from_gpu = [INIT] * C
        self.mbox_op = [0] * C
        self.mbox_seq = [0] * C          # descriptors posted through the mailbox so far
        self.host_seen = [0] * C         # mailbox mode: completions the host has consumed
        # device-side words
        self.gen = [0] * C
        self.bcast = [[(0, 0)] * inst.bcast_depth for _ in range(C)]
        self.dev_done = [0] * C
        self.arrive = [[0] * inst.bcast_depth for _ in range(C)]
        # agents
        self.prod = [[0, -1] for _ in inst.jobs]                      # [next job, ticket or -1]
        self.disp = [0, -1]                                          # [next cluster, ticket or -1]
        # per CTA: [phase, items taken k, held (seq, op)]
        self.cta = [[["poll", 0, (0, 0)] for _ in range(s)] for s in inst.sizes]
        self.logs = [[() for _ in range(s)] for s in inst.sizes]
        self.posted = [() for _ in inst.sizes]   # host's own record: op of descriptor seq = i+1
        self.violations = ()
        self.mutated = False

    def copy(self) -> "State":
        n = State.__new__(State)
        n.inst = self.inst
        for f in ("tail", "done", "to_gpu", "from_gpu", "mbox_op", "mbox_seq", "host_seen",
                  "gen", "dev_done"):
            setattr(n, f, list(getattr(self, f)))
        n.ring = [list(r) for r in self.ring]
        n.bcast = [list(b) for b in self.bcast]
        n.arrive = [list(a) for a in self.arrive]
        n.prod = [list(p) for p in self.prod]
        n.disp = list(self.disp)
        n.cta = [[list(x) for x in cl] for cl in self.cta]
        n.logs = [list(cl) for cl in self.logs]
        n.posted = list(self.posted)
        n.violations = self.violations
        n.mutated = self.mutated
        return n

    def key(self):
        return (tuple(self.tail), tuple(self.done), tuple(self.to_gpu), tuple(self.from_gpu),
                tuple(self.mbox_op), tuple(self.mbox_seq), tuple(self.host_seen), tuple(self.gen),
                tuple(self.dev_done), tuple(map(tuple, self.ring)), tuple(map(tuple, self.bcast)),
                tuple(map(tuple, self.arrive)), tuple(map(tuple, self.prod)), tuple(self.disp),
                tuple(tuple(tuple(x) for x in cl) for cl in self.cta),
                tuple(map(tuple, self.logs)), tuple(self.posted), self.violations, self.mutated)

    # -- helpers ------------------------------------------------------------
    def _flag(self, name):
        if name not in self.violations:
            self.violations = self.violations + (name,)

    def _mut(self, name) -> bool:
        """True once: where the planted mistake `name` fires."""
        if self.inst.mutate == name and not self.mutated:
            self.mutated = True
            return True
        return False

    def producers_done(self) -> bool:
        return all(p[0] == len(j) and p[1] < 0 for p, j in zip(self.prod, self.inst.jobs))

    # -- enabled steps ------------------------------------------------------
    def enabled(self):
        out = []
        inst = self.inst
        R = inst.ring_depth
        for p, (nxt, ticket) in enumerate(self.prod):
            jobs = inst.jobs[p]
            if ticket >= 0:
                out.append(("publish", p))
            elif nxt < len(jobs):
                c = jobs[nxt][0]
                if inst.mode == "ring":
                    full = self.tail[c] - self.done[c] >= R
                    if not full or inst.mutate == "ignore_ring_full":
                        out.append(("ticket", p))
                else:
                    if self.to_gpu[c] == T_NOP and self.from_gpu[c] in (INIT, F_NOP) \
                            and self.host_seen[c] == self.mbox_seq[c]:
                        out.append(("post", p))
        if inst.mode == "mailbox":
            for c in range(len(inst.sizes)):
                if self.from_gpu[c] == FINISHED and self.to_gpu[c] >= T_WORK:
                    out.append(("host_wait", c))
        if self.producers_done():
            c, ticket = self.disp
            if c < len(inst.sizes):
                if inst.mode == "ring":
                    if ticket >= 0:
                        out.append(("publish_exit", 0))
                    elif self.tail[c] - self.done[c] < R:
                        out.append(("ticket_exit", 0))
                elif self.to_gpu[c] == T_NOP and self.from_gpu[c] in (INIT, F_NOP):
                    out.append(("post_exit", 0))
        for c, ctas in enumerate(self.cta):
            for r, (phase, k, held) in enumerate(ctas):
                if phase == "exit":
                    continue
                if self._cta_enabled(c, r, phase, k):
                    out.append(("cta", (c, r)))
        return out

    def _cta_enabled(self, c, r, phase, k) -> bool:
        D = self.inst.bcast_depth
        if phase == "poll":
            if r == 0:
                if self.inst.mode == "ring":
                    return self.ring[c][k % self.inst.ring_depth][0] == k + 1
                # mailbox: new work (or EXIT) while idle, or the host's re-arm to acknowledge
                idle = self.from_gpu[c] in (INIT, F_NOP)
                if idle and self.to_gpu[c] in (T_EXIT,) or (idle and self.to_gpu[c] >= T_WORK):
                    return True
                return self.from_gpu[c] == FINISHED and self.to_gpu[c] == T_NOP
            return self.gen[c] >= k + 1
        if phase == "bcast":
            return self.dev_done[c] >= k + 1 - D or self.inst.mutate == "ignore_bcast_free"
        return True  # run / arrive

    # -- one atomic step ----------------------------------------------------
    def step(self, act) -> None:
        kind, who = act
        inst = self.inst
        R = inst.ring_depth
        if kind == "ticket":
            p = who
            c = inst.jobs[p][self.prod[p][0]][0]
            self.prod[p][1] = self.tail[c]
            self.tail[c] += 1
        elif kind == "publish":
            p = who
            c, op = inst.jobs[p][self.prod[p][0]]
            t = self.prod[p][1]
            self._publish(c, t, op)
            self.prod[p][0] += 1
            self.prod[p][1] = -1
        elif kind == "post":
            p = who
            c, op = inst.jobs[p][self.prod[p][0]]
            self.mbox_seq[c] += 1
            self.mbox_op[c] = op
            self.posted[c] = self.posted[c] + (op,)
            self.to_gpu[c] = T_WORK + op
            self.prod[p][0] += 1
        elif kind == "host_wait":
            c = who
            self.host_seen[c] = self.mbox_seq[c]
            self.to_gpu[c] = T_NOP                    # re-arm
        elif kind == "ticket_exit":
            c = self.disp[0]
            self.disp[1] = self.tail[c]
            self.tail[c] += 1
        elif kind == "publish_exit":
            c = self.disp[0]
            self._publish(c, self.disp[1], EXIT_OP)
            self.disp = [c + 1, -1]
        elif kind == "post_exit":
            c = self.disp[0]
            self.to_gpu[c] = T_EXIT
            self.disp = [c + 1, -1]
        elif kind == "cta":
            self._cta_step(*who)
        else:
            raise ValueError(kind)

    def _publish(self, c, t, op):
        R = self.inst.ring_depth
        # slot t % R last held descriptor t - R + 1, which the master must have taken
        if t >= R and self.cta[c][0][1] < t - R + 1:
            self._flag("slot_overwrite")
        self.ring[c][t % R] = (t + 1, op)
        if op != EXIT_OP:
            # tickets are taken in order, so descriptor t+1 is the (t+1)-th post
            # once every earlier ticket has been published; keep it by index
            rec = list(self.posted[c]) + [None] * max(0, t + 1 - len(self.posted[c]))
            rec[t] = op
            self.posted[c] = tuple(rec)

    def _cta_step(self, c, r):
        inst = self.inst
        S = inst.sizes[c]
        D = inst.bcast_depth
        st = self.cta[c][r]
        phase, k, held = st
        if phase == "poll":
            if r == 0:
                if inst.mode == "ring":
                    held = self.ring[c][k % inst.ring_depth]
                else:
                    if self.from_gpu[c] == FINISHED and self.to_gpu[c] == T_NOP:
                        self.from_gpu[c] = F_NOP          # acknowledge the re-arm
                        return
                    if self.to_gpu[c] == T_EXIT:
                        held = (k + 1, EXIT_OP)
                    else:
                        held = (self.mbox_seq[c], self.to_gpu[c] - T_WORK)
                        self.from_gpu[c] = WORKING
                st[:] = ["bcast", k, held]
            else:
                held = self.bcast[c][k % D]
                if held[1] == EXIT_OP:
                    st[:] = ["exit", k, held]
                else:
                    st[:] = ["run", k, held]
        elif phase == "bcast":          # master relays to the other ranks
            self.bcast[c][k % D] = held
            self.gen[c] = k + 1
            st[:] = ["exit", k, held] if held[1] == EXIT_OP else ["run", k, held]
        elif phase == "run":
            seq, op = held
            smid = inst.smids[c][r]
            if self._mut("wrong_smid"):
                smid = smid + 1000
            if self._mut("wrong_op"):
                op = op + 1
            if not self._mut("skip_share"):
                self.logs[c][r] = self.logs[c][r] + ((seq, op, smid),)
            if self._mut("double_share"):
                self.logs[c][r] = self.logs[c][r] + ((seq, op, smid),)
            st[:] = ["arrive", k, held]
        elif phase == "arrive":
            seq, op = held
            a = self.arrive[c][k % D] + 1
            need = S - 1 if (inst.mutate == "early_complete" and S > 1) else S
            if a >= need and not (a > need):
                # last arrival: every share of `seq` must have been logged by now
                for q in range(S):
                    if not any(e[0] == seq for e in self.logs[c][q]):
                        self._flag("early_complete")
                a = 0 if need == S else a
                self.dev_done[c] = seq
                if inst.mode == "ring":
                    self.done[c] = seq
                else:
                    self.from_gpu[c] = FINISHED
            if a > need:  # the planted early completion left one straggler
                a = 0
            self.arrive[c][k % D] = a
            st[:] = ["poll", k + 1, (0, 0)]

    def terminal(self) -> bool:
        return all(ph == "exit" for cl in self.cta for ph, _, _ in cl)


# -- drivers -----------------------------------------------------------------
def run_random(inst: Instance, seed: int, max_steps: int = 10_000_000) -> State:
    """One interleaving picked by a seeded scheduler."""
    rng = random.Random(seed)
    s = State(inst)
    for _ in range(max_steps):
        if s.terminal():
            return s
        en = s.enabled()
        if not en:
            s._flag("deadlock")
            return s
        s.step(rng.choice(en))
    s._flag("step_limit")
    return s


def explore(inst: Instance, max_states: int = 2_000_000):
    """Every reachable terminal state (depth-first search over distinct states).

    Returns (terminal states, number of distinct states visited).  A state with
    no enabled step that is not terminal is reported with a "deadlock" flag."""
    start = State(inst)
    seen = {start.key()}
    stack = [start]
    terminals = {}
    while stack:
        s = stack.pop()
        if s.terminal():
            terminals[s.key()] = s
            continue
        en = s.enabled()
        if not en:
            d = s.copy()
            d._flag("deadlock")
            terminals[d.key()] = d
            continue
        for act in en:
            n = s.copy()
            n.step(act)
            k = n.key()
            if k not in seen:
                if len(seen) >= max_states:
                    raise RuntimeError("state space larger than max_states")
                seen.add(k)
                stack.append(n)
    return list(terminals.values()), len(seen)


def log_columns(s: State):
    """Flatten the per-rank logs into checker columns."""
    cols = {k: [] for k in ("seq", "cluster", "rank", "smid", "op", "order")}
    for c, cl in enumerate(s.logs):
        for r, log in enumerate(cl):
            for i, (seq, op, smid) in enumerate(log):
                cols["seq"].append(seq)
                cols["cluster"].append(c)
                cols["rank"].append(r)
                cols["smid"].append(smid)
                cols["op"].append(op)
                cols["order"].append(i)
    return cols


def check_state(s: State) -> dict:
    """Checker verdict for one simulated run plus the inline violations."""
    import numpy as np
    from . import check_exec_log

    inst = s.inst
    cols = log_columns(s)
    C = len(inst.sizes)
    n_posted = [len(s.posted[c]) for c in range(C)]
    posted_op = [op for c in range(C) for op in s.posted[c]]
    pinned = [inst.smids[c][r] for c in range(C) for r in range(inst.sizes[c])]
    res = check_exec_log(np.array(cols["seq"], dtype=np.uint64), cols["cluster"], cols["rank"],
                         cols["smid"], cols["op"], cols["order"], inst.sizes, n_posted,
                         pinned_smid=pinned, posted_op=posted_op)
    res["inline"] = list(s.violations)
    res["ok"] = res["violations"] == 0 and not s.violations
    return res
