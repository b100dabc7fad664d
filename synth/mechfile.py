"""Binary mechanism file: the one format every reader in this project parses.

The layout is little-endian:

    char[8]  magic "DLBMECH1"
    int32    nsp, nrx, nelem, n_eff
    f64[nsp] W        molar mass, g/mol
    f64[nsp] cp_a     cp = cp_a + cp_b*T, J/(mol K)
    f64[nsp] cp_b     J/(mol K^2)
    f64[nsp] hf       formation enthalpy at T0 = 298.15 K, J/mol
    f64[nsp] s0       standard entropy at T0 and p0 = 1 atm, J/(mol K)
    i32[nsp*nelem] atoms (species-major; elements C, H, O, N)
    nrx reaction records, each:
        f64 lnA   (A in mol, cm^3, s units of the reaction's order)
        f64 beta  (temperature exponent)
        f64 Ea    (J/mol)
        i32 nr, np, reversible, thirdbody
        i32 ridx[3], rnu[3], pidx[3], pnu[3]   (unused slots are -1 / 0)
    n_eff records of (i32 reaction, i32 species, f64 efficiency): third-body
        efficiencies that differ from 1; every other species counts with 1.
    optional pressure-dependent (fall-off) section:
        char[8] "FALLOFF1", i32 n_fall, then n_fall records of
        i32 reaction, i32 kind (1 Lindemann, 2 Troe with 3 parameters,
        3 Troe with 4), f64 lnA0, beta0, Ea0 (low-pressure limit, same units
        as the high-pressure limit in the reaction record, one order higher),
        f64 a, T3, T1, T2 (Troe parameters; T2 used by kind 3 only).
        A fall-off reaction is a third-body reaction whose [M] (with its
        efficiencies) enters through the reduced pressure instead of
        multiplying the rate.
    optional pressure-dependent Arrhenius (PLOG) section, after the fall-off
    section if both are present:
        char[8] "PLOG0001", i32 n_plog, then n_plog records of
        i32 reaction, i32 npts, npts x (f64 p [Pa], lnA, beta, Ea [J/mol]),
        pressures strictly increasing. The reaction's rate constant at
        pressure p: between the two listed pressures that bracket p, ln k is
        linear in ln p; below the first or above the last listed pressure it
        is that point's Arrhenius form. The reaction record's own lnA, beta,
        Ea are not used. A PLOG reaction is neither third-body nor fall-off.
    optional NASA-7 thermo section (then the cp_a, cp_b, hf, s0 arrays
    above are not used):
        char[8] "NASA7001", then per species 17 f64: Tlow, Tmid, Thigh, the
        low-range coefficients a1..a7 (T < Tmid) and the high-range ones
        (T >= Tmid), with cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4,
        h/(R T) = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T,
        s/R = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7
        (s at p0 = 1 atm, T in K). Outside [Tlow, Thigh] the nearer range's
        polynomials are used as they are.
    The optional sections may appear in any order, each at most once.

Each species appears at most once per side; its integer coefficient is in
rnu / pnu.
"""
from __future__ import annotations

import dataclasses
import struct

import numpy as np

MAGIC = b"DLBMECH1"
ELEMENTS = ("C", "H", "O", "N")
ATOMIC_MASS = np.array([12.011, 1.008, 15.999, 14.007])


@dataclasses.dataclass
class Mechanism:
    W: np.ndarray
    cp_a: np.ndarray
    cp_b: np.ndarray
    hf: np.ndarray
    s0: np.ndarray
    atoms: np.ndarray            # [nsp, 4] int
    lnA: np.ndarray              # [nrx]
    beta: np.ndarray
    Ea: np.ndarray
    reac: list                   # per reaction: list of (species, nu)
    prod: list
    reversible: np.ndarray       # [nrx] int
    thirdbody: np.ndarray        # [nrx] int
    eff: list = dataclasses.field(default_factory=list)  # (rxn, species, eff)
    falloff: list = dataclasses.field(default_factory=list)  # (rxn, kind, lnA0, beta0, Ea0, a, T3, T1, T2)
    plog: list = dataclasses.field(default_factory=list)     # (rxn, [(p_Pa, lnA, beta, Ea), ...])
    nasa: np.ndarray = None      # [nsp, 17] Tlow, Tmid, Thigh, low a1..a7, high a1..a7, or None

    @property
    def nsp(self) -> int:
        return len(self.W)

    @property
    def nrx(self) -> int:
        return len(self.lnA)

    def nu_matrix(self) -> tuple[np.ndarray, np.ndarray]:
        """Reactant and product coefficient matrices, each [nsp, nrx]."""
        nr = np.zeros((self.nsp, self.nrx), dtype=np.int64)
        npd = np.zeros((self.nsp, self.nrx), dtype=np.int64)
        for j, (r, p) in enumerate(zip(self.reac, self.prod)):
            for k, nu in r:
                nr[k, j] += nu
            for k, nu in p:
                npd[k, j] += nu
        return nr, npd


def write_mech(path: str, m: Mechanism) -> None:
    nsp, nrx = m.nsp, m.nrx
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<4i", nsp, nrx, 4, len(m.eff)))
        for arr in (m.W, m.cp_a, m.cp_b, m.hf, m.s0):
            f.write(np.asarray(arr, dtype="<f8").tobytes())
        f.write(np.asarray(m.atoms, dtype="<i4").reshape(-1).tobytes())
        for j in range(nrx):
            r, p = m.reac[j], m.prod[j]
            if not (1 <= len(r) <= 3 and 1 <= len(p) <= 3):
                raise ValueError(f"reaction {j}: 1..3 species per side")
            ridx = [k for k, _ in r] + [-1] * (3 - len(r))
            rnu = [nu for _, nu in r] + [0] * (3 - len(r))
            pidx = [k for k, _ in p] + [-1] * (3 - len(p))
            pnu = [nu for _, nu in p] + [0] * (3 - len(p))
            f.write(struct.pack("<3d", float(m.lnA[j]), float(m.beta[j]), float(m.Ea[j])))
            f.write(struct.pack("<16i", len(r), len(p), int(m.reversible[j]), int(m.thirdbody[j]),
                                *ridx, *rnu, *pidx, *pnu))
        for (j, k, e) in m.eff:
            f.write(struct.pack("<2id", int(j), int(k), float(e)))
        if m.falloff:
            f.write(b"FALLOFF1")
            f.write(struct.pack("<i", len(m.falloff)))
            for rec in m.falloff:
                j, kind = int(rec[0]), int(rec[1])
                if kind not in (1, 2, 3) or not m.thirdbody[j]:
                    raise ValueError(f"fall-off record {rec}: kind 1..3 on a third-body reaction")
                f.write(struct.pack("<2i7d", j, kind, *[float(x) for x in rec[2:9]]))
        if m.plog:
            fall_rx = {int(rec[0]) for rec in m.falloff}
            f.write(b"PLOG0001")
            f.write(struct.pack("<i", len(m.plog)))
            for j, pts in m.plog:
                j = int(j)
                ps = [float(q[0]) for q in pts]
                if (not pts or m.thirdbody[j] or j in fall_rx or min(ps) <= 0
                        or any(b <= a for a, b in zip(ps, ps[1:]))):
                    raise ValueError(f"PLOG record of reaction {j}: increasing positive pressures, "
                                     "not on a third-body or fall-off reaction")
                f.write(struct.pack("<2i", j, len(pts)))
                for q in pts:
                    f.write(struct.pack("<4d", *[float(x) for x in q]))
        if m.nasa is not None:
            nasa = np.asarray(m.nasa, dtype="<f8")
            if nasa.shape != (nsp, 17) or not (nasa[:, 1] > 0).all():
                raise ValueError("NASA-7 data: [nsp, 17] with positive Tmid")
            f.write(b"NASA7001")
            f.write(nasa.tobytes())


def read_mech(path: str) -> Mechanism:
    with open(path, "rb") as f:
        buf = f.read()
    if buf[:8] != MAGIC:
        raise ValueError(f"{path}: not a DLBMECH1 file")
    nsp, nrx, nelem, neff = struct.unpack_from("<4i", buf, 8)
    off = 24
    arrs = []
    for _ in range(5):
        arrs.append(np.frombuffer(buf, dtype="<f8", count=nsp, offset=off).copy())
        off += 8 * nsp
    atoms = np.frombuffer(buf, dtype="<i4", count=nsp * nelem, offset=off).reshape(nsp, nelem).copy()
    off += 4 * nsp * nelem
    lnA, beta, Ea, reac, prod, rev, tb = [], [], [], [], [], [], []
    for _ in range(nrx):
        a, b, e = struct.unpack_from("<3d", buf, off)
        off += 24
        v = struct.unpack_from("<16i", buf, off)
        off += 64
        nr, npd = v[0], v[1]
        lnA.append(a); beta.append(b); Ea.append(e)
        rev.append(v[2]); tb.append(v[3])
        reac.append([(v[4 + i], v[7 + i]) for i in range(nr)])
        prod.append([(v[10 + i], v[13 + i]) for i in range(npd)])
    eff = []
    for _ in range(neff):
        j, k, e = struct.unpack_from("<2id", buf, off)
        off += 16
        eff.append((j, k, e))
    falloff, plog, nasa = [], [], None
    while len(buf) >= off + 8:
        tag = buf[off:off + 8]
        off += 8
        if tag == b"FALLOFF1":
            (nf,) = struct.unpack_from("<i", buf, off)
            off += 4
            for _ in range(nf):
                falloff.append(tuple(struct.unpack_from("<2i7d", buf, off)))
                off += 64
        elif tag == b"PLOG0001":
            (npl,) = struct.unpack_from("<i", buf, off)
            off += 4
            for _ in range(npl):
                j, n = struct.unpack_from("<2i", buf, off)
                off += 8
                pts = [struct.unpack_from("<4d", buf, off + 32 * i) for i in range(n)]
                off += 32 * n
                plog.append((j, [tuple(q) for q in pts]))
        elif tag == b"NASA7001":
            nasa = np.frombuffer(buf, dtype="<f8", count=17 * nsp, offset=off).reshape(nsp, 17).copy()
            off += 8 * 17 * nsp
        else:
            raise ValueError(f"{path}: unknown section {tag!r}")
    return Mechanism(W=arrs[0], cp_a=arrs[1], cp_b=arrs[2], hf=arrs[3], s0=arrs[4], atoms=atoms,
                     lnA=np.array(lnA), beta=np.array(beta), Ea=np.array(Ea), reac=reac, prod=prod,
                     reversible=np.array(rev), thirdbody=np.array(tb), eff=eff, falloff=falloff, plog=plog, nasa=nasa)
