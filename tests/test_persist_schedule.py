"""Persistent heat schedule (csrc/persist.cuh), checked on the host.

The kernel waits, before a unit's step s, for the units that own the R cells beyond each of its
six faces (periodic) to have published step s-1.  This test restates that rule from the source
and checks it:
* the star stencil of Eqs. 5 and 7 reads, along each axis, only cells within R of a unit's
  box.  Every owner of such a cell, other than the unit itself, is among the units waited for.
  This is brute force over extents, tile lengths (short ragged tiles and chunks shorter than
  R included) and radii 1..4;
* a simulation of G CTAs taking units b, b + G, ... in order, step after step, with these
  waits, finishes every step of every unit: there is no deadlock for any G <= the unit count.
"""
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "paper_2406_08923_gb300", "csrc", "persist.cuh")).read()
KSRC = open(os.path.join(ROOT, "paper_2406_08923_gb300", "csrc", "diffusion_f32.cu")).read()


def test_rule_source_is_the_restated_one():
    for text in ("const int ax = threadIdx.x / (2 * R), side = (threadIdx.x / R) & 1, k = threadIdx.x % R + 1;",
                 "const int lo = t * L, hi = min(n, lo + L);",
                 "int cell = side ? hi - 1 + k : lo - k;",
                 "cell = ((cell % n) + n) % n;",
                 "const int o = cell / L;",
                 "if (threadIdx.x < 6 * R) {"):
        assert text in SRC, text
    # the kernel waits from step 1 on, for target epoch + s, and publishes epoch + s + 1
    assert "if (s > 0) ok = wait_face_neighbours<R>(sync, pg, g, t0, t1, t2, base + s, base + 1);" in KSRC
    assert "publish_unit(sync, u, base + s + 1);" in KSRC
    assert "for (int u = blockIdx.x; ok && u < W; u += gridDim.x) {" in KSRC


def waited_owners(t, n, L, R):
    """Tiles along one axis whose flags tile t waits for (the rule of wait_face_neighbours)."""
    lo, hi = t * L, min(n, t * L + L)
    out = set()
    for side in (0, 1):
        for k in range(1, R + 1):
            cell = (hi - 1 + k) if side else (lo - k)
            o = (cell % n) // L
            if o != t:
                out.add(o)
    return out


def read_owners(t, n, L, R):
    """Tiles along one axis that own a cell which the star stencil of tile t reads."""
    lo, hi = t * L, min(n, t * L + L)
    out = set()
    for c in range(lo, hi):
        for a in range(1, R + 1):
            out.add(((c + a) % n) // L)
            out.add(((c - a) % n) // L)
    out.discard(t)
    return out


def test_every_read_owner_is_waited_for():
    checked = 0
    for R in range(1, 5):
        for n in list(range(2 * R + 1, 40)) + [64, 67, 128, 130, 200, 256, 383]:
            for L in sorted({1, 2, 3, 4, 5, 6, 7, 8, 10, 16, 37, 128, n}):
                if L > n:
                    continue
                tiles = (n + L - 1) // L
                for t in range(tiles):
                    need, have = read_owners(t, n, L, R), waited_owners(t, n, L, R)
                    assert need <= have, (R, n, L, t, need - have)
                    checked += 1
    assert checked > 10000


def _simulate(nt, G, nsteps, R, n, L):
    """Round-robin simulation of the persistent kernel's CTAs; returns True if all finish."""
    W = nt[0] * nt[1] * nt[2]
    flag = [0] * W                           # steps published per unit
    pos = [(0, b) for b in range(G)]         # (step, unit) each CTA is at
    def coords(u):
        return u % nt[0], (u // nt[0]) % nt[1], u // (nt[0] * nt[1])
    def unit(q):
        return q[0] + nt[0] * (q[1] + nt[1] * q[2])
    def deps(u):
        t = coords(u)
        out = set()
        for ax in range(3):
            for o in waited_owners(t[ax], n[ax], L[ax], R):
                q = list(t)
                q[ax] = o
                out.add(unit(q))
        return out
    dep = [deps(u) for u in range(W)]
    active = [b < W for b in range(G)]
    while any(active):
        moved = False
        for b in range(G):
            if not active[b]:
                continue
            s, u = pos[b]
            if s > 0 and any(flag[v] < s for v in dep[u]):
                continue  # waits for step s-1 of a neighbour
            flag[u] = s + 1
            moved = True
            u += G
            if u >= W:
                s, u = s + 1, b
            if s >= nsteps:
                active[b] = False
            pos[b] = (s, u)
        if not moved:
            return False
    return all(f == nsteps for f in flag)


def test_schedule_never_deadlocks():
    R = 3
    for n, L in [((256, 256, 256), (128, 8, 37)), ((64, 16, 7), (128, 8, 1)), ((130, 24, 40), (128, 4, 5)),
                 ((512, 128, 64), (128, 8, 5))]:
        nt = tuple((a + b - 1) // b for a, b in zip(n, L))
        W = nt[0] * nt[1] * nt[2]
        for G in sorted({1, 2, 3, W // 3 or 1, W // 2 or 1, W - 1 or 1, W}):
            assert _simulate(nt, G, 4, R, n, L), (n, L, G)

