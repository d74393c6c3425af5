"""Compile-time structure of the hexahedral serendipity element (build step).

Writes refpattern.h for the CUDA kernels: for orders 2, 3, 4 the nonzero pattern
of the nodal derivative matrices D^alpha_ij = d psi_j / d xi_alpha (x_i) (the
flux differences of Eqs. C.34 / D.29 in nodal collocation form), and the nodes on
each face and edge of the reference cube (the supports of the point
evaluations at face and edge points).  Only the pattern is compiled in; the
values still come from the host tables at mesh creation, which check that every
nonzero of their D^alpha lies in this pattern.

The element is the one the host tables build: the unit cube [-1/2, 1/2]^3, the
monomials of superlinear degree <= p-1, nodes = the 8 vertices
(v = ix + 2 iy + 4 iz) then p-2 equidistant nodes inside each of the 12 edges in
edge order (0-3 along xi, 4-7 along eta, 8-11 along zeta).  The Lagrange basis is
found exactly, in rational arithmetic, so that structural zeros are exact.
"""
import itertools
from fractions import Fraction as Fr

EDGE_AXIS = [0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2, 2]
EDGE_FIX = [(-1, -1), (1, -1), (-1, 1), (1, 1)] * 3      # the other two coordinates, in units of 1/2
FACE_AXIS = [0, 0, 1, 1, 2, 2]
FACE_SIDE = [-1, 1, -1, 1, -1, 1]


def exponents(p):
    r = p - 1
    out = []
    for tot in range(0, 3 * r + 1):
        for a, b, c in itertools.product(range(r + 1), repeat=3):
            if a + b + c != tot:
                continue
            if sum(e for e in (a, b, c) if e >= 2) <= r:
                out.append((a, b, c))
    return out


def nodes(p):
    half = Fr(1, 2)
    out = [(Fr(ix) - half, Fr(iy) - half, Fr(iz) - half)
           for iz in range(2) for iy in range(2) for ix in range(2)]
    for e in range(12):
        for s in range(1, p - 1):
            t = -half + Fr(s, p - 1)
            fix = [Fr(f, 2) for f in EDGE_FIX[e]]
            x, q = [], 0
            for a in range(3):
                if a == EDGE_AXIS[e]:
                    x.append(t)
                else:
                    x.append(fix[q])
                    q += 1
            out.append(tuple(x))
    return out


def _inverse(A):
    n = len(A)
    M = [list(row) + [Fr(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [row[n:] for row in M]


def _mono(x, e):
    v = Fr(1)
    for a in range(3):
        v *= x[a] ** e[a]
    return v


def _dmono(x, e, ax):
    if e[ax] == 0:
        return Fr(0)
    v = Fr(e[ax])
    for a in range(3):
        v *= x[a] ** (e[a] - 1 if a == ax else e[a])
    return v


def derivative_pattern(p):
    """[alpha] -> list of (i, j) with D^alpha_ij != 0, by row i then column j."""
    ex, xs = exponents(p), nodes(p)
    N = len(xs)
    C = _inverse([[_mono(x, e) for e in ex] for x in xs])   # C[m][j]
    pat = []
    for ax in range(3):
        ent = []
        for i in range(N):
            dm = [_dmono(xs[i], e, ax) for e in ex]
            for j in range(N):
                if sum(dm[m] * C[m][j] for m in range(N)) != 0:
                    ent.append((i, j))
        pat.append(ent)
    return pat


def face_nodes(p):
    xs = nodes(p)
    return [[i for i, x in enumerate(xs) if x[FACE_AXIS[f]] == Fr(FACE_SIDE[f], 2)] for f in range(6)]


def edge_nodes(p):
    """Nodes on each edge, in node order (the order of the host tables' lists)."""
    xs = nodes(p)
    out = []
    for e in range(12):
        ax = EDGE_AXIS[e]
        fix = [Fr(f, 2) for f in EDGE_FIX[e]]
        on = []
        for i, x in enumerate(xs):
            rest = [x[a] for a in range(3) if a != ax]
            if rest == fix:
                on.append(i)
        out.append(on)
    return out


# Row groups per (zone, variable) of the variable team: a thread computes the rows
# of its group, so fewer groups reuse each loaded 16-byte chunk of F for more
# rows (FP32 FMAs per chunk: about 8 with 4 groups at p = 4, 15 with 2; the
# GB300 SM issues 128 FP32 FMAs per 128 B of shared-memory bandwidth, i.e. 16 per
# chunk) but leave fewer threads for the phase.  Measured (FP32-bulk predictor):
# p = 4, 4 -> 2 groups 27.6 -> 26.1 ms on 1,572,864 zones, 1 group 31.3 ms;
# p = 3, 2 -> 1 group 0.85 -> 0.96 ms on 196,608 zones.
ROW_GROUPS = {2: 1, 3: 2, 4: 2}


def row_groups(p, pat):
    """Contiguous row ranges [RG[g], RG[g+1]) with balanced entry counts over the
    three directions (one group per thread of a zone's variable team)."""
    N = len(nodes(p))
    cnt = [0] * N
    for ax in pat:
        for i, _ in ax:
            cnt[i] += 1
    G = ROW_GROUPS[p]
    tot, rg, acc = sum(cnt), [0], 0
    for i in range(N):
        acc += cnt[i]
        if len(rg) < G and acc >= tot * len(rg) / G:
            rg.append(i + 1)
    rg.append(N)
    assert len(rg) == G + 1
    return rg


def header():
    lines = ["// Generated by paper_1905_02504_gb300/refpattern.py at build time; do not edit.",
             "// Nonzero pattern of the nodal derivative matrices D^alpha and the face / edge",
             "// node lists of the hexahedral serendipity element (orders 2, 3, 4).",
             "#pragma once", "namespace geo {", "template <int P> struct RefPattern;"]
    for p in (2, 3, 4):
        pat = derivative_pattern(p)
        nnz = len(pat[0])
        assert all(len(x) == nnz for x in pat)
        fn, en = face_nodes(p), edge_nodes(p)
        flat = [e for ax in pat for e in ax]
        lines.append("template <> struct RefPattern<%d> {" % p)
        lines.append("  static constexpr int NNZ = %d, NFN = %d, NEN = %d;" % (nnz, len(fn[0]), len(en[0])))
        lines.append("  // entry e of direction alpha: row I[alpha * NNZ + e], column J[alpha * NNZ + e]")
        lines.append("  static constexpr unsigned char I[%d] = {%s};" % (len(flat), ", ".join(str(i) for i, _ in flat)))
        lines.append("  static constexpr unsigned char J[%d] = {%s};" % (len(flat), ", ".join(str(j) for _, j in flat)))
        lines.append("  static constexpr unsigned char FN[%d] = {%s};" % (6 * len(fn[0]), ", ".join(str(i) for f in fn for i in f)))
        lines.append("  static constexpr unsigned char EN[%d] = {%s};" % (12 * len(en[0]), ", ".join(str(i) for e in en for i in e)))
        rg = row_groups(p, pat)
        eg = [[sum(1 for i, _ in ax if i < r) for r in rg] for ax in pat]
        lines.append("  // row groups [RG[g], RG[g+1]) and their entry ranges [EG[alpha][g], EG[alpha][g+1])")
        lines.append("  static constexpr int G = %d;" % (len(rg) - 1))
        lines.append("  static constexpr int RG[%d] = {%s};" % (len(rg), ", ".join(map(str, rg))))
        lines.append("  static constexpr int EG[3][%d] = {%s};" % (len(rg), ", ".join("{%s}" % ", ".join(map(str, e)) for e in eg)))
        lines.append("};")
    lines.append("}  // namespace geo")
    return "\n".join(lines) + "\n"


def write(path):
    text = header()
    try:
        if open(path).read() == text:
            return path
    except OSError:
        pass
    with open(path, "w") as f:
        f.write(text)
    return path


if __name__ == "__main__":
    import sys
    print(header() if len(sys.argv) < 2 else write(sys.argv[1]))
