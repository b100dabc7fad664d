"""CHEMKIN-format mechanism text to the binary mechanism file (and back).

The subset read: ELEMENTS (C, H, O, N), SPECIES, THERMO with NASA-7 entries
in the fixed-column layout (four lines per species: name, element counts,
Tlow, Thigh and Tmid on the first; a1..a7 of the high range, then a1..a7 of
the low range, five 15-character fields per line), and REACTIONS: a
reaction line `reactants <=> products  A  beta  Ea` ('=' and '<=>'
reversible, '=>' irreversible; integer coefficients written before the
species, `+M` third body, `(+M)` fall-off) followed by auxiliary lines with
`LOW / A0 beta0 Ea0 /`, `TROE / a T3 T1 [T2] /`, `PLOG / p[atm] A beta Ea /`,
`DUPLICATE` and third-body efficiencies `SPECIES / value /`. Units on the
REACTIONS line: CAL/MOLE (default), KCAL/MOLE, JOULES/MOLE, KJOULES/MOLE,
KELVINS for Ea; MOLES (default) for A. Comments start at '!'.

Not read (ValueError): other elements, fractional coefficients, more than
three molecules on a side, reactions whose elements do not balance, explicit reverse parameters (REV), SRI and
Chebyshev forms, third bodies that are a named species ((+H2O)), several
Arrhenius terms at one PLOG pressure, MOLECULES units.

    python -m synth.chemkin mech.inp [thermo.dat] out.bin
"""
from __future__ import annotations

import math
import re
import sys

import numpy as np

from .mechfile import ATOMIC_MASS, ELEMENTS, Mechanism, write_mech

R = 8.314462618
T0 = 298.15
_EA = {"CAL/MOLE": 4.184, "KCAL/MOLE": 4184.0, "JOULES/MOLE": 1.0, "KJOULES/MOLE": 1000.0, "KELVINS": R}


def _strip(text: str) -> list[str]:
    return [ln.split("!", 1)[0].rstrip() for ln in text.splitlines()]


_KEYWORDS = {"ELEMENTS": "ELEM", "ELEM": "ELEM", "SPECIES": "SPEC", "SPEC": "SPEC", "THERMO": "THER",
             "THER": "THER", "REACTIONS": "REAC", "REAC": "REAC"}


def _blocks(lines: list[str]) -> dict:
    """Lines of each keyword block (ELEM, SPEC, THER, REAC), keyword line
    first. A block ends at END or, except THERMO, at the next keyword."""
    out, cur = {}, None
    for ln in lines:
        up = ln.strip().upper()
        first = up.split()[0] if up else ""
        if first == "END" and cur is not None:
            cur = None
            continue
        if first in _KEYWORDS and (cur is None or cur != "THER"):
            cur = _KEYWORDS[first]
            out[cur] = [ln]
            continue
        if cur is not None:
            out[cur].append(ln)
    return out


def _num(s: str) -> float:
    return float(s.strip().replace("D", "E").replace("d", "e"))


def parse_thermo(lines: list[str], species: list[str]) -> dict:
    """NASA-7 entries by species name: (Tlow, Tmid, Thigh, low a1..a7, high a1..a7, atoms)."""
    body = [ln for ln in lines[1:] if ln.strip()]
    gT = None
    if body and len(body[0].split()) in (3, 4) and not body[0].rstrip().endswith("1"):
        gT = [_num(x) for x in body[0].split()[:3]]
        body = body[1:]
    out = {}
    i = 0
    while i + 3 < len(body):
        l1, l2, l3, l4 = (body[i + j].ljust(80) for j in range(4))
        if l1[79] != "1":
            i += 1
            continue
        name = l1[:18].split()[0]
        atoms = {}
        for f in range(4):
            el, cnt = l1[24 + 5 * f:26 + 5 * f].strip().upper(), l1[26 + 5 * f:29 + 5 * f].strip()
            if el and el != "0" and cnt:
                atoms[el] = atoms.get(el, 0) + int(round(float(cnt)))
        Tlow, Thigh = _num(l1[45:55]), _num(l1[55:65])
        Tmid = _num(l1[65:73]) if l1[65:73].strip() else (gT[1] if gT else 1000.0)
        co = [_num(ln[15 * j:15 * j + 15]) for ln in (l2, l3) for j in range(5)] + \
             [_num(l4[15 * j:15 * j + 15]) for j in range(4)]
        high, low = co[0:7], co[7:14]
        out[name.upper()] = (Tlow, Tmid, Thigh, low, high, atoms)
        i += 4
    missing = [s for s in species if s.upper() not in out]
    if missing:
        raise ValueError(f"no thermo data for {missing}")
    return out


_SIDE_COEF = re.compile(r"^(\d+)?([A-Za-z(].*)$")


def _side(text: str, idx: dict) -> tuple[list, bool]:
    terms = [t for t in text.split("+") if t]
    sp, tb = {}, False
    for t in terms:
        if t.upper() == "M":
            tb = True
            continue
        mt = _SIDE_COEF.match(t)
        if not mt:
            raise ValueError(f"cannot read term {t!r}")
        nu = int(mt.group(1)) if mt.group(1) else 1
        name = mt.group(2).upper()
        if name not in idx:
            raise ValueError(f"unknown species {name!r}")
        sp[idx[name]] = sp.get(idx[name], 0) + nu
    return sorted(sp.items()), tb


def parse_reactions(lines: list[str], idx: dict):
    head = lines[0].upper().split()[1:]
    ea = 4.184
    for w in head:
        if w in _EA:
            ea = _EA[w]
        elif w == "MOLECULES":
            raise ValueError("MOLECULES units are not read")
        elif w != "MOLES":
            raise ValueError(f"unknown REACTIONS unit {w!r}")
    rx = []
    for ln in lines[1:]:
        s = ln.strip()
        if not s:
            continue
        up = s.upper()
        if "/" in s or up.startswith("DUP"):
            if not rx:
                raise ValueError(f"auxiliary line before any reaction: {s!r}")
            r = rx[-1]
            if up.startswith("DUP"):
                continue
            parts = re.findall(r"([^/\s][^/]*?)\s*/([^/]*)/", s)
            for key, val in parts:
                key = key.strip().upper()
                vals = [_num(v) for v in val.split()]
                if key == "LOW":
                    r["low"] = (math.log(vals[0]), vals[1], vals[2] * ea)
                elif key == "TROE":
                    r["troe"] = vals
                elif key == "PLOG":
                    p = vals[0] * 101325.0
                    if any(abs(q[0] - p) <= 1e-12 * p for q in r["plog"]):
                        raise ValueError("several Arrhenius terms at one PLOG pressure are not read")
                    if not vals[1] > 0:
                        raise ValueError("PLOG A must be positive")
                    r["plog"].append((p, math.log(vals[1]), vals[2], vals[3] * ea))
                elif key in ("REV", "SRI", "CHEB", "PCHEB", "TCHEB", "LT", "RLT", "HIGH", "FORD", "RORD"):
                    raise ValueError(f"{key} is not read")
                elif key in idx:
                    r["eff"].append((idx[key], vals[0]))
                else:
                    raise ValueError(f"unknown auxiliary keyword or species {key!r}")
            continue
        tok = s.split()
        if len(tok) < 4:
            raise ValueError(f"cannot read reaction line {s!r}")
        A, beta, Ea = _num(tok[-3]), _num(tok[-2]), _num(tok[-1])
        eq = "".join(tok[:-3])
        fall = "(+M)" in eq.upper()
        if fall:
            eq = re.sub(r"\(\+M\)", "", eq, flags=re.I)
        if re.search(r"\(\+[^)]*\)", eq):
            raise ValueError("a named third body is not read")
        for arrow, rev in (("<=>", 1), ("=>", 0), ("=", 1)):
            if arrow in eq:
                lhs, rhs = eq.split(arrow, 1)
                break
        else:
            raise ValueError(f"no arrow in {eq!r}")
        reac, tb1 = _side(lhs, idx)
        prod, tb2 = _side(rhs, idx)
        if tb1 != tb2:
            raise ValueError(f"+M on one side only in {eq!r}")
        if fall and tb1:
            raise ValueError(f"both (+M) and +M in {eq!r}")
        if not A > 0:
            raise ValueError(f"A must be positive in {eq!r}")
        rx.append(dict(reac=reac, prod=prod, rev=rev, tb=int(tb1 or fall), fall=fall, lnA=math.log(A), beta=beta,
                       Ea=Ea * ea, eff=[], plog=[], low=None, troe=None))
    return rx


def read_chemkin(mech_text: str, thermo_text: str | None = None) -> Mechanism:
    blocks = _blocks(_strip(mech_text))
    el_lines = blocks.get("ELEM", [])
    els = " ".join([" ".join(el_lines[0].split()[1:])] + el_lines[1:]).upper().split() if el_lines else []
    for e in els:
        if e not in ELEMENTS:
            raise ValueError(f"element {e} is not read (C, H, O, N only)")
    spec_lines = blocks.get("SPEC")
    if not spec_lines:
        raise ValueError("no SPECIES block")
    species = (" ".join(spec_lines[0].split()[1:]) + " " + " ".join(spec_lines[1:])).split()
    species = [s.upper() for s in species]
    idx = {s: i for i, s in enumerate(species)}
    ther = blocks.get("THER")
    if thermo_text is not None:
        tb = _blocks(_strip(thermo_text)).get("THER") or (["THERMO"] + _strip(thermo_text))
        ther = tb
    if ther is None:
        raise ValueError("no THERMO data")
    th = parse_thermo(ther, species)
    nsp = len(species)
    atoms = np.zeros((nsp, 4), dtype=np.int64)
    nasa = np.zeros((nsp, 17))
    for k, s in enumerate(species):
        Tlow, Tmid, Thigh, low, high, at = th[s]
        for e, c in at.items():
            if e not in ELEMENTS:
                raise ValueError(f"species {s}: element {e} is not read (C, H, O, N only)")
            atoms[k, ELEMENTS.index(e)] += c
        nasa[k] = [Tlow, Tmid, Thigh, *low, *high]
    W = atoms @ ATOMIC_MASS

    def cp_h_s(k, T):
        c = nasa[k, 3:10] if T < nasa[k, 1] else nasa[k, 10:17]
        cp = R * (c[0] + c[1] * T + c[2] * T ** 2 + c[3] * T ** 3 + c[4] * T ** 4)
        h = R * T * (c[0] + c[1] * T / 2 + c[2] * T ** 2 / 3 + c[3] * T ** 3 / 4 + c[4] * T ** 4 / 5 + c[5] / T)
        s_ = R * (c[0] * math.log(T) + c[1] * T + c[2] * T ** 2 / 2 + c[3] * T ** 3 / 3 + c[4] * T ** 4 / 4 + c[6])
        return cp, h, s_

    # the linear-thermo fields are informative only when NASA-7 data are present
    cp_a = np.array([cp_h_s(k, 1000.0)[0] for k in range(nsp)])
    hf = np.array([cp_h_s(k, T0)[1] for k in range(nsp)])
    s0 = np.array([cp_h_s(k, T0)[2] for k in range(nsp)])
    rx = parse_reactions(blocks.get("REAC", ["REACTIONS"]), idx)
    eff, falloff, plog = [], [], []
    for j, r in enumerate(rx):
        for side in (r["reac"], r["prod"]):
            if sum(nu for _, nu in side) > 3 or len(side) > 3:
                raise ValueError(f"reaction {j}: more than three molecules on a side")
        bal = sum(nu * atoms[k] for k, nu in r["reac"]) - sum(nu * atoms[k] for k, nu in r["prod"])
        if np.any(bal != 0):
            raise ValueError(f"reaction {j}: elements not balanced")
        if r["eff"] and not r["tb"]:
            raise ValueError(f"reaction {j}: efficiencies without a third body")
        for k, e in r["eff"]:
            eff.append((j, k, e))
        if r["fall"]:
            if r["low"] is None:
                raise ValueError(f"reaction {j}: (+M) without LOW")
            t = r["troe"]
            kind = 1 if t is None else (2 if len(t) == 3 else 3)
            a, T3, T1, T2 = (t + [0.0] * (4 - len(t))) if t else (0.0, 1.0, 1.0, 0.0)
            falloff.append((j, kind, *r["low"], a, T3, T1, T2))
        if r["plog"]:
            if r["tb"]:
                raise ValueError(f"reaction {j}: PLOG with a third body")
            plog.append((j, sorted(r["plog"])))
    return Mechanism(W=W, cp_a=cp_a, cp_b=np.zeros(nsp), hf=hf, s0=s0, atoms=atoms,
                     lnA=np.array([r["lnA"] for r in rx]), beta=np.array([r["beta"] for r in rx]),
                     Ea=np.array([r["Ea"] for r in rx]), reac=[r["reac"] for r in rx], prod=[r["prod"] for r in rx],
                     reversible=np.array([r["rev"] for r in rx]), thirdbody=np.array([r["tb"] for r in rx]),
                     eff=eff, falloff=falloff, plog=plog, nasa=nasa)


def _f15(x: float) -> str:
    return f"{x:15.8E}"


def write_chemkin(m: Mechanism, names: list[str] | None = None) -> str:
    """CHEMKIN text of a mechanism with NASA-7 thermo (m.nasa): the inverse of
    read_chemkin up to the 9 significant digits of the thermo fields. Ea is
    written in J/mol, PLOG pressures in atm."""
    if m.nasa is None:
        raise ValueError("write_chemkin needs NASA-7 data (synth.nasa7_of_linear gives them for linear cp)")
    names = names or [f"S{k}" for k in range(m.nsp)]
    out = ["ELEMENTS", " ".join(ELEMENTS), "END", "SPECIES", " ".join(names), "END", "THERMO ALL",
           "   200.000  1000.000  6000.000"]
    for k, nm in enumerate(names):
        els = "".join(f"{e:<2}{int(c):>3}" for e, c in zip(ELEMENTS, m.atoms[k]) if c) or "C   0"
        els = els.ljust(20)[:20]
        Tlow, Tmid, Thigh = m.nasa[k, :3]
        low, high = m.nasa[k, 3:10], m.nasa[k, 10:17]
        out.append(f"{nm:<18}{'':6}{els}G{Tlow:10.3f}{Thigh:10.3f}{Tmid:8.2f}      1")
        co = list(high) + list(low)
        out.append("".join(_f15(x) for x in co[0:5]) + "    2")
        out.append("".join(_f15(x) for x in co[5:10]) + "    3")
        out.append("".join(_f15(x) for x in co[10:14]) + "                   4")
    out += ["END", "REACTIONS JOULES/MOLE MOLES"]
    fall = {int(r[0]): r for r in m.falloff}
    plog = {int(j): pts for j, pts in m.plog}
    effs = {}
    for j, k, e in m.eff:
        effs.setdefault(int(j), []).append((int(k), e))

    def side(lst):
        return "+".join((f"{nu}" if nu > 1 else "") + names[k] for k, nu in lst)

    for j in range(m.nrx):
        arrow = "<=>" if m.reversible[j] else "=>"
        tb = ""
        if j in fall:
            tb = "(+M)"
        elif m.thirdbody[j]:
            tb = "+M"
        eq = side(m.reac[j]) + tb + arrow + side(m.prod[j]) + tb
        out.append(f"{eq}  {math.exp(m.lnA[j])!r}  {float(m.beta[j])!r}  {float(m.Ea[j])!r}")
        if j in fall:
            r = fall[j]
            out.append(f"  LOW / {math.exp(r[2])!r} {float(r[3])!r} {float(r[4])!r} /")
            if r[1] == 2:
                out.append(f"  TROE / {float(r[5])!r} {float(r[6])!r} {float(r[7])!r} /")
            elif r[1] == 3:
                out.append(f"  TROE / {float(r[5])!r} {float(r[6])!r} {float(r[7])!r} {float(r[8])!r} /")
        if j in plog:
            for p, lnA, beta, Ea in plog[j]:
                out.append(f"  PLOG / {p / 101325.0!r} {math.exp(lnA)!r} {float(beta)!r} {float(Ea)!r} /")
        if j in effs:
            out.append("  " + " ".join(f"{names[k]}/{e!r}/" for k, e in effs[j]))
    out.append("END")
    return "\n".join(out) + "\n"


def main(argv):
    if len(argv) not in (3, 4):
        print(__doc__)
        return 2
    thermo = open(argv[2]).read() if len(argv) == 4 else None
    m = read_chemkin(open(argv[1]).read(), thermo)
    write_mech(argv[-1], m)
    print(f"{argv[-1]}: {m.nsp} species, {m.nrx} reactions, {len(m.falloff)} fall-off, {len(m.plog)} PLOG")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
