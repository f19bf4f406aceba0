"""CPU checks of what the loader hands to the kernel, by emulation.

* The executable program (dumped with pc_debug_program) is run by a
  test-side emulator of the warp-uniform stack machine -- 32-lane warps,
  FP32 values, branch skipping only when no live lane needs a branch, loop
  exit once every live lane latched -- on the oracle's simulated paths, and
  must reproduce the oracle's per-path payoffs.
* The date-ordered bridge schedule (pc_debug_bridge), replayed with its
  per-level Philox block caches on the oracle's normals, must reproduce the
  oracle's breadth-first array-form bridge exactly.
"""
import numpy as np
import pytest

import paper_2108_03076_gb300 as pc
import workloads as W
from oracle import il_text, mc, paths as opaths
from oracle.paths import Market

OPS = ["END", "CONST", "MODEL", "PAYOFF", "TIME", "NOW", "NEGF", "NOT", "ADDF", "SUBF", "MULF",
       "DIVF", "MAXF", "MINF", "LTF", "LEF", "EQF", "ADDI", "SUBI", "MULI", "MAXI", "MINI", "LTI",
       "LEI", "EQI", "AND", "OR", "ADDFK", "SUBFK", "MULFK", "DIVFK", "MAXFK", "MINFK", "LTFK",
       "LEFK", "EQFK", "RSUBFK", "RDIVFK", "RLTFK", "RLEFK", "MODEL_MULK", "MODEL_DIVK", "IF",
       "ELSE", "SEL", "LOOP", "LTEST", "LLATCH", "LNEXT", "LEND", "LRED", "LANY", "LSTEPK", "LOOPANY"]
OP = {n: i for i, n in enumerate(OPS)}
LF_K, LF_T0, LF_DONE, LF_RES, LF_NEWLY = range(5)


def f32(bits):
    return np.array([bits], np.uint32).view(np.float32)[0]


def _cmp(code, v, k):
    return {1: v < k, 2: v <= k, 3: k < v, 4: k <= v}[code]


def run_warp(code, pool, S, sval, disc, n_hist, now, live):
    """Emulate one warp: S[lane, label, ordinal 0..n] float32; returns float32 [32]."""
    L = len(live)
    slots = {}
    tos = np.zeros(L, np.float32)
    sp, pc_, t0 = 0, 0, 0
    steps = 0

    def ld(s):
        return slots.get(s, np.zeros(L, np.float32)).copy()

    def st(s, v):
        slots[s] = np.asarray(v, np.float32).copy()

    def asi(v):
        return np.asarray(v, np.float32).view(np.int32)

    def asf(v):
        return np.asarray(v, np.int32).view(np.float32)

    def push(v):
        nonlocal sp, tos
        st(sp, tos)
        sp += 1
        tos = np.asarray(v, np.float32).copy()

    def fused(ins, t0_):
        opa_, b_, c_, e_ = (int(x) for x in ins)
        A_ = opa_ >> 8
        bs_ = b_ - (1 << 32) if b_ >= (1 << 31) else b_
        o = bs_ + t0_ - now
        n = ((A_ >> 8) & 3) + 1
        kind, cmpc = (A_ >> 2) & 3, (A_ >> 4) & 7
        kk = f32(e_)
        v = None
        for i in range(n):
            lab = (A_ >> (10 + 2 * i)) & 3
            sv = (S[:, lab, o] if o > 0 else np.full(L, sval[o + n_hist][lab])).astype(np.float32)
            if kind == 1:
                sv = sv * pool[c_ + i]
            elif kind == 2:
                sv = sv / pool[c_ + i]
            if OPS[opa_ & 0xFF] == "LANY":
                pi = _cmp(cmpc, sv, kk)
                v = pi if v is None else ((v & pi) if A_ & 1 else (v | pi))
            else:
                rop = A_ & 3
                v = sv if v is None else (np.fmin(v, sv) if rop == 0 else np.fmax(v, sv) if rop == 1
                                          else (v + sv).astype(np.float32))
        if OPS[opa_ & 0xFF] == "LANY":
            return asf(v.astype(np.int32))
        if cmpc:
            return asf(_cmp(cmpc, v, kk).astype(np.int32))
        return np.asarray(v, np.float32)

    while True:
        steps += 1
        assert steps < 10 ** 7, "runaway program"
        opa, b, c, e = (int(x) for x in code[pc_])
        bs = b - (1 << 32) if b >= (1 << 31) else b          # operand b as int32
        op, A = opa & 0xFF, opa >> 8
        name = OPS[op]
        kb = f32(b)
        if name == "END":
            return tos
        if name == "CONST":
            push(np.full(L, np.uint32(b)).view(np.float32)); pc_ += 1
        elif name in ("MODEL", "MODEL_MULK", "MODEL_DIVK"):
            o = bs + t0 - now
            v = S[:, A, o] if o > 0 else np.full(L, sval[o + n_hist][A], np.float32)
            v = v.astype(np.float32)
            if name == "MODEL_MULK":
                v = v * f32(c)
            elif name == "MODEL_DIVK":
                v = v / f32(c)
            push(v); pc_ += 1
        elif name in ("LRED", "LANY"):
            push(fused(code[pc_], t0)); pc_ += 1
        elif name == "LOOPANY":
            F, lit = A & 0xFF, pool[A >> 8]
            desc = code[pc_ + 1]
            done, res = ~live, np.zeros(L, np.float32)
            allv = False
            for kk in range(b + 1):
                cnd = asi(fused(desc, t0 + kk)) != 0
                nw = cnd & ~done
                res = np.where(nw, lit, res).astype(np.float32)
                done = done | nw
                allv = bool(np.all(done))
                if allv:
                    break
            if allv:
                push(res); pc_ = e
            else:
                st(F + LF_T0, asf(np.full(L, t0, np.int32)))
                st(F + LF_DONE, asf(done.astype(np.int32)))
                st(F + LF_RES, res)
                t0 += b
                pc_ += 2
        elif name == "LRED_UNUSED":
            o = bs + t0 - now
            n = ((A >> 8) & 3) + 1
            kind, cmpc = (A >> 2) & 3, (A >> 4) & 7
            kk = f32(e)
            v = None
            for i in range(n):
                lab = (A >> (10 + 2 * i)) & 3
                sv = (S[:, lab, o] if o > 0 else np.full(L, sval[o + n_hist][lab])).astype(np.float32)
                if kind == 1:
                    sv = sv * pool[c + i]
                elif kind == 2:
                    sv = sv / pool[c + i]
                if name == "LANY":
                    pi = _cmp(cmpc, sv, kk)
                    v = pi if v is None else ((v & pi) if A & 1 else (v | pi))
                else:
                    rop = A & 3
                    v = sv if v is None else (np.fmin(v, sv) if rop == 0 else np.fmax(v, sv) if rop == 1
                                              else (v + sv).astype(np.float32))
            if name == "LANY":
                v = asf(v.astype(np.int32))
            elif cmpc:
                v = asf(_cmp(cmpc, v, kk).astype(np.int32))
            push(np.asarray(v, np.float32)); pc_ += 1
        elif name == "LSTEPK":
            F, pidx = A & 0xFF, A >> 8
            cnd = asi(tos)
            sp -= 1
            tos = ld(sp)
            done = asi(ld(F + LF_DONE))
            nw = (cnd != 0) & (done == 0)
            lit = pool[pidx]
            st(F + LF_RES, np.where(nw, lit, ld(F + LF_RES)))
            st(F + LF_DONE, asf(np.where(nw, 1, done).astype(np.int32)))
            t0e = int(asi(ld(F + LF_T0))[0])
            if np.all(asi(ld(F + LF_DONE)) != 0):
                t0 = t0e
                push(ld(F + LF_RES)); pc_ = e
            else:
                k = int(asi(ld(F + LF_K))[0])
                if k == b:
                    t0 = t0e + k; pc_ += 1
                else:
                    k += 1
                    st(F + LF_K, asf(np.full(L, k, np.int32)))
                    t0 = t0e + k; pc_ = c
        elif name == "PAYOFF":
            o = bs + t0 - now
            v = np.float32(f32(c) * np.float32(disc[o + n_hist]))
            push(np.full(L, -v if A else v, np.float32)); pc_ += 1
        elif name == "TIME":
            push(asf(np.full(L, bs + t0, np.int32))); pc_ += 1
        elif name == "NOW":
            push(asf(np.full(L, now, np.int32))); pc_ += 1
        elif name == "NEGF":
            tos = -tos; pc_ += 1
        elif name == "NOT":
            tos = asf(asi(tos) ^ 1); pc_ += 1
        elif name in ("ADDF", "SUBF", "MULF", "DIVF", "MAXF", "MINF", "LTF", "LEF", "EQF"):
            bb, aa = tos, ld(sp - 1)
            sp -= 1
            with np.errstate(all="ignore"):
                r = {"ADDF": lambda: aa + bb, "SUBF": lambda: aa - bb, "MULF": lambda: aa * bb,
                     "DIVF": lambda: aa / bb, "MAXF": lambda: np.fmax(aa, bb),
                     "MINF": lambda: np.fmin(aa, bb),
                     "LTF": lambda: asf((aa < bb).astype(np.int32)),
                     "LEF": lambda: asf((aa <= bb).astype(np.int32)),
                     "EQF": lambda: asf((aa == bb).astype(np.int32))}[name]()
            tos = np.asarray(r, np.float32); pc_ += 1
        elif name in ("ADDI", "SUBI", "MULI", "MAXI", "MINI", "LTI", "LEI", "EQI", "AND", "OR"):
            bb, aa = asi(tos), asi(ld(sp - 1))
            sp -= 1
            r = {"ADDI": aa + bb, "SUBI": np.where(aa > bb, aa - bb, 0), "MULI": aa * bb,
                 "MAXI": np.maximum(aa, bb), "MINI": np.minimum(aa, bb), "LTI": aa < bb,
                 "LEI": aa <= bb, "EQI": aa == bb, "AND": aa & bb, "OR": aa | bb}[name]
            tos = asf(np.asarray(r).astype(np.int32)); pc_ += 1
        elif name.endswith("FK"):
            x, k = tos, kb
            with np.errstate(all="ignore"):
                r = {"ADDFK": lambda: x + k, "SUBFK": lambda: x - k, "MULFK": lambda: x * k,
                     "DIVFK": lambda: x / k, "MAXFK": lambda: np.fmax(x, k),
                     "MINFK": lambda: np.fmin(x, k),
                     "LTFK": lambda: asf((x < k).astype(np.int32)),
                     "LEFK": lambda: asf((x <= k).astype(np.int32)),
                     "EQFK": lambda: asf((x == k).astype(np.int32)),
                     "RSUBFK": lambda: k - x, "RDIVFK": lambda: k / x,
                     "RLTFK": lambda: asf((k < x).astype(np.int32)),
                     "RLEFK": lambda: asf((k <= x).astype(np.int32))}[name]()
            tos = np.asarray(r, np.float32); pc_ += 1
        elif name == "IF":
            cnd = asi(tos) != 0
            if np.any(live & cnd):
                pc_ += 1
            else:
                push(np.zeros(L, np.float32)); pc_ = c
        elif name == "ELSE":
            cnd = asi(ld(sp - 1)) != 0
            if np.any(live & ~cnd):
                pc_ += 1
            else:
                push(np.zeros(L, np.float32)); pc_ = c
        elif name == "SEL":
            th, cnd = ld(sp - 1), asi(ld(sp - 2))
            sp -= 2
            tos = np.where(cnd != 0, th, tos).astype(np.float32); pc_ += 1
        elif name == "LOOP":
            st(A + LF_K, asf(np.zeros(L, np.int32)))
            st(A + LF_T0, asf(np.full(L, t0, np.int32)))
            st(A + LF_DONE, asf((~live).astype(np.int32)))
            st(A + LF_RES, np.zeros(L, np.float32)); pc_ += 1
        elif name == "LTEST":
            cnd = asi(tos)
            sp -= 1
            tos = ld(sp)
            nw = (cnd != 0) & (asi(ld(A + LF_DONE)) == 0)
            st(A + LF_NEWLY, asf(nw.astype(np.int32)))
            pc_ = pc_ + 1 if np.any(nw) else c
        elif name == "LLATCH":
            v = tos
            sp -= 1
            tos = ld(sp)
            nw = asi(ld(A + LF_NEWLY)) != 0
            st(A + LF_RES, np.where(nw, v, ld(A + LF_RES)))
            st(A + LF_DONE, asf(np.where(nw, 1, asi(ld(A + LF_DONE))).astype(np.int32))); pc_ += 1
        elif name == "LNEXT":
            t0e = int(asi(ld(A + LF_T0))[0])
            if np.all(asi(ld(A + LF_DONE)) != 0):
                t0 = t0e
                push(ld(A + LF_RES)); pc_ = e
            else:
                k = int(asi(ld(A + LF_K))[0])
                if k == b:
                    t0 = t0e + k; pc_ += 1
                else:
                    k += 1
                    st(A + LF_K, asf(np.full(L, k, np.int32)))
                    t0 = t0e + k; pc_ = c
        elif name == "LEND":
            done = asi(ld(A + LF_DONE)) != 0
            tos = np.where(done, ld(A + LF_RES), tos).astype(np.float32)
            t0 = int(asi(ld(A + LF_T0))[0]); pc_ += 1
        else:
            raise AssertionError(name)


def emulate(text, spec, tparams, n, seed, p1=0, p2=1):
    w, k = pc.pc_assemble(text)
    code, pool = pc.pc_debug_program(w, k, tparams, p1, p2)
    mk = Market(**vars(spec))
    S = opaths.simulate(mk, seed, 0, np.arange(n, dtype=np.uint64)).astype(np.float32)
    H = len(mk.history)
    sval = [list(mk.history[H - 1 - i]) for i in range(H)] + [list(mk.S0)]   # ordinal -H..0
    disc = [mk.disc(o + mk.now) for o in range(-H, mk.n + 1)]
    out = np.zeros(n, np.float32)
    for w0 in range(0, n, 32):
        idx = np.arange(w0, w0 + 32)
        live = idx < n
        Sw = S[np.minimum(idx, n - 1)]
        out[w0:w0 + 32][: live.sum()] = run_warp(code, pool, Sw, sval, disc, H, mk.now, live)[live]
    return out.astype(np.float64)


from cases import CASES  # noqa: E402


@pytest.mark.parametrize("name", list(CASES))
def test_program_emulation_matches_oracle(name):
    text, tp, spec, notional = CASES[name]
    n = 96 + 7 if spec.n >= 100 else 512 + 7
    got = emulate(text, spec, tp, n, 0x51)
    ref, marg = mc.payoffs(il_text.parse(text), Market(**vars(spec)),
                           {f"${i}": v for i, v in enumerate(tp)}, 0, 1, n, 0x51, with_margins=True)
    tol = 2e-6 * np.maximum(np.abs(ref), notional)
    bad = (np.abs(got - ref) > tol) & (marg >= 1e-5)
    assert not bad.any(), (name, np.nonzero(bad)[0][:5], got[bad][:5], ref[bad][:5])


# ---------------------------------------------------------------------------
# Bridge schedule
# ---------------------------------------------------------------------------

GRIDS = [([365], 1), ([1, 2], 2), ([5, 10, 15], 3), (list(range(1, 9)), 1), (list(range(1, 13)), 4),
         (list(range(1, 366)), 3), (list(range(1, 366)), 1), ([3, 9, 27, 81, 243, 729], 2),
         (list(range(7, 3651, 7)), 4), (list(range(1, 101)), 2), (list(range(1, 1001)), 3)]


@pytest.mark.parametrize("days,d", GRIDS)
def test_date_ordered_bridge_matches_array_form(days, d):
    n = len(days)
    corr = np.eye(d).tolist()
    dops, ops = pc.pc_debug_bridge([1.0] * d, [0.2] * d, corr, 0.0, days)
    P = 8
    z = opaths.normals(99, 0, np.arange(P, dtype=np.uint64), n * d)        # [p, m]
    tau = np.concatenate([[0.0], np.asarray(days, float) / 365.0])
    nodes = opaths.bridge_schedule(tau)
    want = opaths.bridge_apply(nodes, np.moveaxis(opaths.node_normals(
        nodes, d, 99, 0, np.arange(P, dtype=np.uint64)), 2, 1), n)        # [p, i, o]
    rank = opaths.generation_order(nodes)
    wl, wr, sd = (ops[:, k].view(np.float32).astype(np.float64) for k in range(3))
    cur = np.zeros((P, d))
    stack = []
    got = np.zeros((P, d, n + 1))
    nodes_seen = []
    for t in range(1, n + 1):
        a, b = dops[t], dops[t + 1]
        if a == b:
            cur = stack.pop()
        for k in range(a, b):
            j, fl = int(ops[k, 3]), int(ops[k, 4]) >> 16
            nodes_seen.append(j)
            # op k is the k-th node the walk computes: normals d k .. d k + d - 1
            assert rank[j] == k
            zz = z[:, d * k:d * k + d]
            if fl & 1:
                nw = np.float64(sd[k]) * zz
            else:
                nw = wl[k] * cur + wr[k] * stack[-1] + sd[k] * zz
            if k + 1 < b:
                stack.append(nw)
            else:
                cur = nw
        got[:, :, t] = cur
        assert int(ops[dops[t + 1] - 1, 5]) == t if b > a else True
    # float32 weights vs FP64 weights: agree to float rounding
    np.testing.assert_allclose(got, want, rtol=0, atol=3e-6 * max(1.0, np.sqrt(tau[-1])))
    # every bridge node is visited once
    assert sorted(nodes_seen) == list(range(n))


def test_fused_ops_are_emitted_for_workloads():
    """The worst-of and barrier programs use the fused multi-asset ops."""
    names = []
    for text, tp in [(W.autocall_text([1.0, 2.0, 0.5]), []),
                     (W.barrier_ladder_text([1.0, 1.0, 1.0]), [365])]:
        w, k = pc.pc_assemble(text)
        code, pool = pc.pc_debug_program(w, k, tp)
        names.append([OPS[int(x) & 0xFF] for x in code[:, 0]])
    assert names[0].count("LRED") >= 10 and "MINF" not in names[0]
    assert "LANY" in names[1] and "LOOPANY" in names[1] and "LSTEPK" not in names[1]
