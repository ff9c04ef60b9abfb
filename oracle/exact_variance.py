"""Exact moments of the AIRPF likelihood estimate on finite HMMs -- TEST INFRASTRUCTURE.

Three independent computations, used to pin each other and the sampling code:

* ``forward_z``: the forward algorithm, Z = p(y_{1:T}) exactly (the target of
  Theorem 1's lack of bias, E[Z^N] = Z).
* ``pair_moments``: E[Z^N] and E[(Z^N)^2] from a recursion over pairs of
  islands, written from Theorem 3 and Lemmas 2-3 (Section 3.3).  The state is
  P_kl(x, x') = E[W^k W^l 1{block_k = x, block_l = x'}] over ordered island
  blocks x in X^M.  Islands k != l move independently given the past; k = l is
  the collision case C_1 (one block, kept on the diagonal).  The internal
  resampling kernel is R_t of eq. (22); an interaction stage with alpha = A_s
  mixes the pair over {k, k xor b} x {l, l xor b} with weights 1/4 (eqs.
  (28)-(29)).  With radix r (A_s = I (x) r^-1 1_r (x) I, m a power of r) a stage
  mixes the pair over grp(k) x grp(l) with weights 1/r^2: islands k != l draw
  their group members independently, so when grp(k) = grp(l) they land on the
  same member (the collision term) with probability sum_c W_c^2 / (sum_c W_c)^2.
  The island at the end of step q is the island at the start of step q+1.  Only
  fixed interaction (always / never, and m = 1) closes this recursion; adaptive
  interaction needs the brute force below.
* ``brute_force_moments``: enumerates every random outcome of Algorithm 1
  (prior, mutation, resampling, island choices, adaptive ENF tests) in exact
  rational arithmetic for tiny sizes.

Time indexing as elsewhere: x_0 ~ pi_0, then for t = 1..T mutate, weight with
y_t, resample and interact.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def toy_model(p_stay=0.75, p_correct=0.75):
    """Binary HMM of Section 4.1: (pi0[2], K[2,2], g(y) -> g[2])."""
    pi0 = np.array([0.5, 0.5])
    K = np.array([[p_stay, 1 - p_stay], [1 - p_stay, p_stay]])

    def g(y):
        y = int(round(float(y)))
        return np.array([p_correct if x == y else 1 - p_correct for x in (0, 1)])
    return pi0, K, g


def forward_z(pi0, K, gs):
    """log Z = log p(y_{1:T}) by the forward algorithm; gs[t-1] = g_t over X."""
    pred = np.asarray(pi0, dtype=np.float64) @ K
    logz = 0.0
    for g in gs:
        a = pred * g
        z = a.sum()
        logz += np.log(z)
        pred = (a / z) @ K
    return logz


def _blocks(M, nx):
    return list(itertools.product(range(nx), repeat=M))


def _group(k, s, radix):
    """The islands of k's group at stage s (base-radix digit s-1 of k varied), member order."""
    bits = int(round(np.log2(radix)))
    stride = 1 << (bits * (s - 1))
    base = k & ~((radix - 1) * stride)
    return [base + c * stride for c in range(radix)]


def pair_moments(pi0, K, gs, m, M, interact, radix=2):
    """(E[Z^N_T], E[(Z^N_T)^2]) for AIRPF with m islands of M particles and
    fixed interaction (interact=True: every stage uses A_s; False: alpha = I);
    radix r: stages over groups of r islands (m a power of r)."""
    pi0 = np.asarray(pi0, dtype=np.float64)
    nx = len(pi0)
    blocks = _blocks(M, nx)
    nb = len(blocks)
    bidx = np.array(blocks)                             # [nb, M]
    pb = np.prod(pi0[bidx], axis=1)                     # prior of a block
    Kb = np.ones((nb, nb))
    for i in range(M):
        Kb *= K[bidx[:, i]][:, bidx[:, i]]              # K^{(x)M}(x, y)
    S = int(round(np.log2(m))) // int(round(np.log2(radix)))
    r2 = float(radix * radix)

    F = np.tile(pb, (m, 1))                            # E[W^k 1{x}]
    P = np.zeros((m, m, nb, nb))
    for k in range(m):
        for l in range(m):
            P[k, l] = np.diag(pb) if k == l else np.outer(pb, pb)

    for g in gs:
        g = np.asarray(g, dtype=np.float64)
        # mutation K_t^{(x)M}: independent for k != l, once for k = l
        F = F @ Kb
        for k in range(m):
            for l in range(m):
                if k == l:
                    P[k, k] = np.diag(np.diag(P[k, k]) @ Kb)
                else:
                    P[k, l] = Kb.T @ P[k, l] @ Kb
        # weighting by gbar(x) = M^-1 sum_i g(x_i)
        gx = g[bidx]                                    # [nb, M]
        gbar = gx.mean(axis=1)
        F = F * gbar
        P = P * np.outer(gbar, gbar)
        # internal multinomial resampling: R[x, z] = prod_j sum_{i: x_i = z_j} g(x_i) / sum_i g(x_i)
        R = np.ones((nb, nb))
        tot = gx.sum(axis=1)
        for j in range(M):
            match = (bidx[:, None, :] == bidx[None, :, j][:, :, None])   # [x, z, i]
            R *= (match * gx[:, None, :]).sum(axis=2) / tot[:, None]
        F = F @ R
        for k in range(m):
            for l in range(m):
                if k == l:
                    P[k, k] = np.diag(np.diag(P[k, k]) @ R)
                else:
                    P[k, l] = R.T @ P[k, l] @ R
        # interaction stages with alpha_s = A_s
        if interact:
            for s in range(1, S + 1):
                Fn = np.empty_like(F)
                Pn = np.empty_like(P)
                for k in range(m):
                    gk = _group(k, s, radix)
                    Fn[k] = sum(F[a] for a in gk) / radix
                    for l in range(m):
                        gl = _group(l, s, radix)
                        acc = sum(P[a, b] for a in gk for b in gl)
                        Pn[k, l] = acc / r2 if k != l else np.diag(acc.sum(axis=1) / r2)
                F, P = Fn, Pn
    ez = F.sum() / m
    ez2 = P.sum() / (m * m)
    return float(ez), float(ez2)


def brute_force_moments(p_stay, p_correct, ys, m, M, mode, tau=Fraction(1), radix=2):
    """Exact (E[Z], E[Z^2]) as Fractions by enumerating all outcomes of
    Algorithm 1 on the binary HMM.  mode: 0 never, 1 always, 2 adaptive with
    the strict test ENF < tau; radix r: stages over groups of r islands, each
    island drawing one member of its group with probability proportional to
    the weights.  Tiny sizes only (m*M <= 4, T <= 3)."""
    ps, pc = Fraction(p_stay), Fraction(p_correct)
    tau = Fraction(tau)
    S = int(round(np.log2(m))) // int(round(np.log2(radix)))
    N = m * M
    # state: (blocks: tuple of m tuples of M values, weights: tuple of m Fractions) -> prob
    dist = {}
    for xs in itertools.product((0, 1), repeat=N):
        blocks = tuple(tuple(xs[k * M:(k + 1) * M]) for k in range(m))
        key = (blocks, tuple(Fraction(1) for _ in range(m)))
        dist[key] = dist.get(key, 0) + Fraction(1, 2 ** N)

    def add(d, key, p):
        d[key] = d.get(key, 0) + p

    for y in ys:
        y = int(round(float(y)))
        g = {x: (pc if x == y else 1 - pc) for x in (0, 1)}
        # mutation: every particle stays w.p. p_stay
        nd = {}
        for (blocks, W), p in dist.items():
            flat = [v for b in blocks for v in b]
            for flips in itertools.product((0, 1), repeat=N):
                q = p
                new = []
                for v, f in zip(flat, flips):
                    q *= (1 - ps) if f else ps
                    new.append(1 - v if f else v)
                nb = tuple(tuple(new[k * M:(k + 1) * M]) for k in range(m))
                add(nd, (nb, W), q)
        dist = nd
        # weighting and internal resampling, island by island
        nd = {}
        for (blocks, W), p in dist.items():
            Wn = tuple(W[k] * sum(g[v] for v in blocks[k]) / M for k in range(m))
            per_island = []
            for k in range(m):
                tot = sum(g[v] for v in blocks[k])
                opts = {}
                for anc in itertools.product(range(M), repeat=M):
                    q = Fraction(1)
                    for a in anc:
                        q *= g[blocks[k][a]] / tot
                    add(opts, tuple(blocks[k][a] for a in anc), q)
                per_island.append(list(opts.items()))
            for combo in itertools.product(*per_island):
                q = p
                for _, qq in combo:
                    q *= qq
                add(nd, (tuple(b for b, _ in combo), Wn), q)
        dist = nd
        # interaction stages
        for s in range(1, S + 1):
            nd = {}
            for (blocks, W), p in dist.items():
                if mode == 0:
                    interact = False
                elif mode == 1:
                    interact = True
                else:
                    s1 = sum(W) / m
                    s2 = sum(w * w for w in W) / m
                    enf = (s1 * s1 / s2) if s2 > 0 else Fraction(0)
                    interact = enf < tau
                if not interact:
                    add(nd, (blocks, W), p)
                    continue
                groups = [_group(k, s, radix) for k in range(m)]
                Wn = tuple(sum(W[a] for a in groups[k]) / radix for k in range(m))
                choices = []
                for k in range(m):
                    tot = sum(W[a] for a in groups[k])
                    # every weight zero: the last member (the rule of the sampling code)
                    choices.append([(a, W[a] / tot if tot > 0 else Fraction(int(a == groups[k][-1])))
                                    for a in groups[k]])
                for combo in itertools.product(*choices):
                    q = p
                    for _, qq in combo:
                        q *= qq
                    if q == 0:
                        continue
                    add(nd, (tuple(blocks[c] for c, _ in combo), Wn), q)
            dist = nd
    ez = sum(p * (sum(W) / m) for (_, W), p in dist.items())
    ez2 = sum(p * (sum(W) / m) ** 2 for (_, W), p in dist.items())
    return ez, ez2
