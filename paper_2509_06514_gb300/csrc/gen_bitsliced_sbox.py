#!/usr/bin/env python3
"""Generates bs_sbox.cuh: the AES S-box (FIPS-197 §5.1.1) as a boolean circuit on bit-slices,
for the bitsliced AES engine of the calibration kernel (aes_bench.cu).

Construction (a composite-field inversion, the standard route to a small S-box circuit):
  * GF(2^8) of AES (modulus x^8 + x^4 + x^3 + x + 1) is isomorphic to GF(16)[y]/(y^2 + y + lam)
    with GF(16) = GF(2)[z]/(z^4 + z + 1) and lam in GF(16) chosen so that y^2 + y + lam has no
    root in GF(16). The isomorphism sends x to a root g of the AES modulus in the tower field;
    it is linear over GF(2) (an 8 x 8 bit matrix M).
  * In the tower field, a = a1 y + a0 has inverse (a1 y + (a0 + a1)) / D with
    D = lam a1^2 + a1 a0 + a0^2 in GF(16) (a * (a1 y + a0 + a1) = D, using y^2 = y + lam).
  * S(x) = A inv(x) + 0x63 (A the affine matrix), so S = (A M^-1) inv_tower(M x) + 0x63: an input
    linear map, three GF(16) products, one GF(16) inversion, an output linear map.
Linear maps become XOR networks with shared pairs (Paar's greedy method); GF(16) products are
the schoolbook AND-XOR sums reduced mod z^4 + z + 1; the GF(16) inverse is written per output
bit as a two-way choice on the top input bit between two 3-input functions (each one LOP3).
The generator picks, among all valid (lam, g), the one with the fewest XORs in the two linear
maps, and checks the emitted circuit against the S-box on all 256 inputs before writing.

    python paper_2509_06514_gb300/csrc/gen_bitsliced_sbox.py   # rewrites bs_sbox.cuh beside it
"""
from __future__ import annotations

import os

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "bs_sbox.cuh")


# ---- fields -------------------------------------------------------------------------------

def gf256_mul(a: int, b: int) -> int:
    """Product in GF(2^8) modulo x^8 + x^4 + x^3 + x + 1 (FIPS-197 §4.2)."""
    p = 0
    for _ in range(8):
        if b & 1:
            p ^= a
        hi = a & 0x80
        a = (a << 1) & 0xFF
        if hi:
            a ^= 0x1B
        b >>= 1
    return p


def gf256_inv(a: int) -> int:
    return 0 if a == 0 else next(y for y in range(1, 256) if gf256_mul(a, y) == 1)


def sbox_table() -> list[int]:
    """S(x) = affine(inverse(x)), FIPS-197 §5.1.1: b'_i = b_i + b_(i+4) + b_(i+5) + b_(i+6) + b_(i+7) + c_i."""
    out = []
    for x in range(256):
        v = gf256_inv(x)
        s = 0
        for i in range(8):
            bit = ((v >> i) ^ (v >> ((i + 4) % 8)) ^ (v >> ((i + 5) % 8)) ^ (v >> ((i + 6) % 8)) ^
                   (v >> ((i + 7) % 8)) ^ (0x63 >> i)) & 1
            s |= bit << i
        out.append(s)
    return out


def gf16_mul(a: int, b: int) -> int:
    """Product in GF(16) = GF(2)[z] / (z^4 + z + 1)."""
    p = 0
    for i in range(4):
        if (b >> i) & 1:
            p ^= a << i
    for k in (6, 5, 4):
        if (p >> k) & 1:
            p ^= 0b10011 << (k - 4)
    return p


def gf16_inv(a: int) -> int:
    return 0 if a == 0 else next(y for y in range(1, 16) if gf16_mul(a, y) == 1)


def tower_mul(a: int, b: int, lam: int) -> int:
    """(a1 y + a0)(b1 y + b0) with y^2 = y + lam; a1 in the high nibble."""
    a1, a0, b1, b0 = a >> 4, a & 15, b >> 4, b & 15
    hh = gf16_mul(a1, b1)
    c1 = hh ^ gf16_mul(a1, b0) ^ gf16_mul(a0, b1)
    c0 = gf16_mul(hh, lam) ^ gf16_mul(a0, b0)
    return (c1 << 4) | c0


def tower_pow(a: int, e: int, lam: int) -> int:
    r = 1
    for _ in range(e):
        r = tower_mul(r, a, lam)
    return r


# ---- GF(2) linear algebra (matrices as lists of row bit masks: out bit r = parity(row_r & x)) ----

def apply(mat: list[int], x: int) -> int:
    return sum(((bin(row & x).count("1") & 1) << r) for r, row in enumerate(mat))


def mat_from_columns(cols: list[int]) -> list[int]:
    """Matrix whose column i (image of input bit i) is cols[i]."""
    return [sum(((cols[i] >> r) & 1) << i for i in range(8)) for r in range(8)]


def mat_inv(mat: list[int]) -> list[int]:
    n = len(mat)
    rows = [(mat[r], 1 << r) for r in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if (rows[r][0] >> c) & 1)
        rows[c], rows[piv] = rows[piv], rows[c]
        for r in range(n):
            if r != c and (rows[r][0] >> c) & 1:
                rows[r] = (rows[r][0] ^ rows[c][0], rows[r][1] ^ rows[c][1])
    return [rows[r][1] for r in range(n)]


def mat_mul(a: list[int], b: list[int]) -> list[int]:
    """a * b (apply b first)."""
    cols = [apply(a, apply(b, 1 << i)) for i in range(8)]
    return mat_from_columns(cols)


def affine_matrix() -> list[int]:
    """The linear part of the S-box's affine map: output bit i = b_i + b_(i+4) + ... + b_(i+7)."""
    rows = []
    for i in range(8):
        row = 0
        for k in (0, 4, 5, 6, 7):
            row |= 1 << ((i + k) % 8)
        rows.append(row)
    return rows


# ---- circuit building ------------------------------------------------------------------------

class Circuit:
    """Straight-line code over named signals; ops are ('xor', a, b), ('and', a, b),
    ('fn3', (a, b, c), truth) and ('mux', sel, one, zero)."""

    def __init__(self):
        self.ops: list[tuple[str, tuple]] = []
        self.n = 0

    def new(self, op: str, *args) -> str:
        name = f"t{self.n}"
        self.n += 1
        self.ops.append((name, (op,) + args))
        return name

    def xor(self, a, b):
        return self.new("xor", a, b)

    def and_(self, a, b):
        return self.new("and", a, b)


def xor_network(c: Circuit, inputs: list[str], rows: list[int]) -> list[str]:
    """Outputs parity(row & inputs) for each row, sharing pairs greedily (Paar). A row with no
    bit gives the signal '0'."""
    sig = list(inputs)
    rows = list(rows)
    while True:
        best, pair = 0, None
        for i in range(len(sig)):
            for j in range(i + 1, len(sig)):
                cnt = sum(1 for r in rows if (r >> i) & 1 and (r >> j) & 1)
                if cnt > best:
                    best, pair = cnt, (i, j)
        if best < 2:
            break
        i, j = pair
        sig.append(c.xor(sig[i], sig[j]))
        k = len(sig) - 1
        rows = [(r ^ (1 << i) ^ (1 << j) | (1 << k)) if ((r >> i) & 1 and (r >> j) & 1) else r for r in rows]
    outs = []
    for r in rows:
        terms = [sig[i] for i in range(len(sig)) if (r >> i) & 1]
        if not terms:
            outs.append("0")
            continue
        acc = terms[0]
        for t in terms[1:]:
            acc = c.xor(acc, t)
        outs.append(acc)
    return outs


def gf16_mul_circuit(c: Circuit, a: list[str], b: list[str]) -> list[str]:
    """a * b in GF(16), bit lists LSB first: products a_i b_j reduced mod z^4 + z + 1."""
    terms: list[list[str]] = [[] for _ in range(4)]
    for i in range(4):
        for j in range(4):
            p = c.and_(a[i], b[j])
            v = 1 << (i + j)
            # reduce z^(i+j)
            for k in (6, 5, 4):
                if (v >> k) & 1:
                    v ^= 0b10011 << (k - 4)
            for k in range(4):
                if (v >> k) & 1:
                    terms[k].append(p)
    out = []
    for k in range(4):
        acc = terms[k][0]
        for t in terms[k][1:]:
            acc = c.xor(acc, t)
        out.append(acc)
    return out


def gf16_inv_circuit(c: Circuit, d: list[str]) -> list[str]:
    """Inverse in GF(16) (0 -> 0): each output bit is d3 ? f1(d0, d1, d2) : f0(d0, d1, d2)."""
    out = []
    for k in range(4):
        t1 = t0 = 0
        for v in range(8):
            t0 |= ((gf16_inv(v) >> k) & 1) << v
            t1 |= ((gf16_inv(v | 8) >> k) & 1) << v
        f1 = c.new("fn3", (d[0], d[1], d[2]), t1)
        f0 = c.new("fn3", (d[0], d[1], d[2]), t0)
        out.append(c.new("mux", d[3], f1, f0))
    return out


def gf16_lin_rows(f) -> list[int]:
    """Rows (over 4 input bits) of a GF(2)-linear map on GF(16)."""
    return [sum(((f(1 << i) >> r) & 1) << i for i in range(4)) for r in range(4)]


def build(lam: int, g: int):
    # isomorphism M: AES bit i (x^i) -> g^i in the tower field
    M = mat_from_columns([tower_pow(g, i, lam) for i in range(8)])
    Minv = mat_inv(M)
    OUTM = mat_mul(affine_matrix(), Minv)
    c = Circuit()
    x = [f"x{i}" for i in range(8)]
    t = xor_network(c, x, M)                       # tower representation: t[0..3] = a0, t[4..7] = a1
    a0, a1 = t[:4], t[4:]
    # D = lam a1^2 + a0^2 + a1 a0: the linear part as one XOR network over (a0, a1)
    sq = gf16_lin_rows(lambda v: gf16_mul(v, v))
    lsq = gf16_lin_rows(lambda v: gf16_mul(lam, gf16_mul(v, v)))
    lin_rows = [sq[r] | (lsq[r] << 4) for r in range(4)]
    lin = xor_network(c, a0 + a1, lin_rows)
    prod = gf16_mul_circuit(c, a1, a0)
    dd = [lin[r] if prod[r] == "0" else (prod[r] if lin[r] == "0" else c.xor(lin[r], prod[r])) for r in range(4)]
    di = gf16_inv_circuit(c, dd)
    s01 = [c.xor(a0[r], a1[r]) for r in range(4)]
    r1 = gf16_mul_circuit(c, a1, di)
    r0 = gf16_mul_circuit(c, s01, di)
    y = xor_network(c, r0 + r1, OUTM)              # A * M^-1 * inverse, before the constant 0x63
    return c, y, M, OUTM


def evaluate(c: Circuit, outs: list[str], xval: int) -> int:
    env = {f"x{i}": (xval >> i) & 1 for i in range(8)}
    env["0"] = 0
    for name, op in c.ops:
        k = op[0]
        if k == "xor":
            env[name] = env[op[1]] ^ env[op[2]]
        elif k == "and":
            env[name] = env[op[1]] & env[op[2]]
        elif k == "fn3":
            a, b, cc = (env[s] for s in op[1])
            env[name] = (op[2] >> (a | (b << 1) | (cc << 2))) & 1
        elif k == "mux":
            env[name] = env[op[2]] if env[op[1]] else env[op[3]]
    return sum(env[o] << i for i, o in enumerate(outs)) ^ 0x63


def fn3_expr(ins, truth) -> str:
    """A 3-input function as a sum (XOR) of minterm ANDs; the compiler folds any expression of
    three inputs into one LOP3."""
    a, b, cc = ins
    terms = []
    for v in range(8):
        if (truth >> v) & 1:
            lits = [(a if v & 1 else f"~{a}"), (b if v & 2 else f"~{b}"), (cc if v & 4 else f"~{cc}")]
            terms.append("(" + " & ".join(lits) + ")")
    return " | ".join(terms) if terms else "0u"


def emit(c: Circuit, outs: list[str], lam: int, g: int, n_and: int, n_xor: int) -> str:
    lines = []
    for name, op in c.ops:
        k = op[0]
        if k == "xor":
            e = f"{op[1]} ^ {op[2]}"
        elif k == "and":
            e = f"{op[1]} & {op[2]}"
        elif k == "fn3":
            e = fn3_expr(op[1], op[2])
        else:
            e = f"({op[1]} & {op[2]}) | (~{op[1]} & {op[3]})"
        lines.append(f"    const uint32_t {name} = {e};")
    body = "\n".join(lines)
    res = "\n".join(f"    y{i} = {'~' if (0x63 >> i) & 1 else ''}{o};" for i, o in enumerate(outs))
    return f'''// bs_sbox.cuh — GENERATED by gen_bitsliced_sbox.py (do not edit): the AES S-box (FIPS-197
// §5.1.1) as a circuit on bit-slices. x0..x7 are bits 0..7 (LSB first) of the input byte of 32
// independent instances (one per bit of each word); y0..y7 receive the output bits.
// Composite field GF(16)[y]/(y^2 + y + {lam}), GF(16) = GF(2)[z]/(z^4 + z + 1), isomorphism x -> {g:#04x};
// {n_and} ANDs, {n_xor} XORs and 8 GF(16)-inverse lookups of 3 inputs before the compiler fuses
// them into 3-input logic operations. Checked against the S-box on all 256 inputs.
#pragma once

#include <cstdint>

#define IMPIR_BS_SBOX(x0, x1, x2, x3, x4, x5, x6, x7, y0, y1, y2, y3, y4, y5, y6, y7) \\
    do {{                                                                                \\
{chr(10).join(l + " " * max(1, 86 - len(l)) + chr(92) for l in (body + chr(10) + res).split(chr(10)))}
    }} while (0)
'''


def main():
    table = sbox_table()
    best = None
    for lam in range(1, 16):
        if any(gf16_mul(y, y) ^ y ^ lam == 0 for y in range(16)):
            continue  # y^2 + y + lam has a root: not a field extension
        for g in range(2, 256):
            # g must be a root of the AES modulus in the tower field
            v = tower_pow(g, 8, lam) ^ tower_pow(g, 4, lam) ^ tower_pow(g, 3, lam) ^ g ^ 1
            if v:
                continue
            c, y, M, OUTM = build(lam, g)
            cost = len(c.ops)
            if best is None or cost < best[0]:
                best = (cost, lam, g)
    cost, lam, g = best
    c, y, M, OUTM = build(lam, g)
    for xv in range(256):
        assert evaluate(c, y, xv) == table[xv], (xv, evaluate(c, y, xv), table[xv])
    n_and = sum(1 for _, op in c.ops if op[0] == "and")
    n_xor = sum(1 for _, op in c.ops if op[0] == "xor")
    src = emit(c, y, lam, g, n_and, n_xor)
    with open(OUT, "w") as f:
        f.write(src)
    print(f"lam={lam} g={g:#04x}: {len(c.ops)} ops ({n_and} and, {n_xor} xor), checked on 256 inputs -> {OUT}")


if __name__ == "__main__":
    main()
