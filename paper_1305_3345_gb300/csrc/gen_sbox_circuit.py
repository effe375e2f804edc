"""Generates sbox_circuit.cuh: the AES S-box (FIPS-197 section 5.1.1) as a
straight-line circuit of AND/XOR/NOT gates on 32-bit words, for the bitsliced
cipher (each word holds one bit of 32 independent S-box inputs).

Construction (composite-field inversion, as in the compact S-box designs of
Satoh et al. and Canright):

* GF(2^8) is rebuilt as a tower GF(((2^2)^2)^2):
  GF(4)   = GF(2)[w]/(w^2 + w + 1),
  GF(16)  = GF(4)[y]/(y^2 + y + nu),
  GF(256) = GF(16)[z]/(z^2 + z + lam),
  with nu, lam chosen so that each quadratic is irreducible.
* The isomorphism from the AES field GF(2)[x]/(x^8+x^4+x^3+x+1) is the linear
  map sending x to a root beta of the AES polynomial in the tower.
* For a = a1 z + a0 (a1, a0 in GF(16)):
  a^-1 = (a1 z + (a1 + a0)) * D^-1,  D = a1^2 lam + a1 a0 + a0^2 in GF(16),
  and the same formula one level down inverts D in GF(16); in GF(4) the
  inverse is the square.
* Multiplications use the three-product (Karatsuba) form; squarings and
  constant scalings are linear.
* S(x) = A * M^-1 * inv(M * x) + 0x63, with A the affine matrix and M the
  isomorphism; the two linear maps at either end are folded into the XOR
  network.

Every signal is kept as a linear form (a set of wires XORed together) until an
AND gate or an output needs it; the XOR network that computes all those forms
is then built with the greedy shared-pair heuristic of Paar ("Optimized
arithmetic for Reed-Solomon encoders", 1997).  The generator tries every
(nu, lam, beta) and keeps the smallest circuit, checks it on all 256 inputs
against the S-box computed from its definition, and writes the header.

Usage: python gen_sbox_circuit.py [--check]   (--check: compare with the
committed header instead of writing it; exit 1 on a difference)
"""
import itertools
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "sbox_circuit.cuh")


# ---------------------------------------------------------------- fields

def aes_mul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        if a & 0x100:
            a ^= 0x11B
        b >>= 1
    return r


def aes_sbox():
    """FIPS-197 5.1.1: multiplicative inverse (0 -> 0), then the affine map."""
    inv = [0] * 256
    for a in range(1, 256):
        for b in range(1, 256):
            if aes_mul(a, b) == 1:
                inv[a] = b
                break
    s = []
    for a in range(256):
        b = inv[a]
        c = 0
        for i in range(8):
            bit = ((b >> i) ^ (b >> ((i + 4) % 8)) ^ (b >> ((i + 5) % 8)) ^ (b >> ((i + 6) % 8))
                   ^ (b >> ((i + 7) % 8)) ^ (0x63 >> i)) & 1
            c |= bit << i
        s.append(c)
    return s


def gf4_mul(a, b):
    a1, a0, b1, b0 = a >> 1, a & 1, b >> 1, b & 1
    hi = (a1 & b1) ^ (a1 & b0) ^ (a0 & b1)
    lo = (a1 & b1) ^ (a0 & b0)
    return (hi << 1) | lo


def make_tower(nu, lam):
    def gf16_mul(a, b):
        a1, a0, b1, b0 = a >> 2, a & 3, b >> 2, b & 3
        p11 = gf4_mul(a1, b1)
        hi = gf4_mul(a1, b0) ^ gf4_mul(a0, b1) ^ p11
        lo = gf4_mul(p11, nu) ^ gf4_mul(a0, b0)
        return (hi << 2) | lo

    def gf256_mul(a, b):
        a1, a0, b1, b0 = a >> 4, a & 15, b >> 4, b & 15
        p11 = gf16_mul(a1, b1)
        hi = gf16_mul(a1, b0) ^ gf16_mul(a0, b1) ^ p11
        lo = gf16_mul(p11, lam) ^ gf16_mul(a0, b0)
        return (hi << 4) | lo

    return gf16_mul, gf256_mul


def irreducible_quadratic(mul, c, size):
    """t^2 + t + c has no root in the field of the given size."""
    return all(mul(r, r) ^ r ^ c for r in range(size))


def tower_choices():
    for nu in range(1, 4):
        if not irreducible_quadratic(gf4_mul, nu, 4):
            continue
        gf16_mul, _ = make_tower(nu, 0)
        for lam in range(1, 16):
            if not irreducible_quadratic(gf16_mul, lam, 16):
                continue
            _, mul = make_tower(nu, lam)
            for beta in range(2, 256):
                p = [1]
                for _ in range(8):
                    p.append(mul(p[-1], beta))
                if p[8] ^ p[4] ^ p[3] ^ p[1] ^ p[0] == 0:
                    yield nu, lam, beta, p[:8]


def mat_from_columns(cols):
    """8x8 GF(2) matrix (rows as bit masks over input bits) from the images of
    the basis vectors."""
    return [sum(((cols[j] >> i) & 1) << j for j in range(8)) for i in range(8)]


def mat_apply(m, v):
    return sum((bin(m[i] & v).count("1") & 1) << i for i in range(8))


def mat_inverse(m):
    rows = [(m[i], 1 << i) for i in range(8)]
    for c in range(8):
        piv = next(r for r in range(c, 8) if (rows[r][0] >> c) & 1)
        rows[c], rows[piv] = rows[piv], rows[c]
        for r in range(8):
            if r != c and (rows[r][0] >> c) & 1:
                rows[r] = (rows[r][0] ^ rows[c][0], rows[r][1] ^ rows[c][1])
    return [rows[i][1] for i in range(8)]


# ---------------------------------------------------------------- symbolic core

class Core:
    """Symbolic evaluation of the tower inversion on linear forms (frozensets
    of wire names); every AND gate is recorded with its two input forms."""

    def __init__(self, nu, lam):
        self.nu, self.lam = nu, lam
        self.ands = []  # (name, lin_a, lin_b)

    @staticmethod
    def add(a, b):
        return a ^ b

    def gate_and(self, a, b):
        name = f"g{len(self.ands)}"
        self.ands.append((name, a, b))
        return frozenset([name])

    # GF(4): (hi, lo) of linear forms
    def g4_add(self, a, b):
        return (a[0] ^ b[0], a[1] ^ b[1])

    def g4_sq(self, a):                       # (a1 w + a0)^2 = a1 w + (a1 + a0)
        return (a[0], a[0] ^ a[1])

    def g4_scale(self, a, c):
        if c == 0:
            return (frozenset(), frozenset())
        if c == 1:
            return a
        if c == 2:                            # * w
            return (a[0] ^ a[1], a[0])
        return (a[1], a[0] ^ a[1])            # * w^2 = w + 1

    def g4_mul(self, a, b):
        p11 = self.gate_and(a[0], b[0])
        p00 = self.gate_and(a[1], b[1])
        pss = self.gate_and(a[0] ^ a[1], b[0] ^ b[1])
        return (pss ^ p00, p11 ^ p00)

    # GF(16): (hi, lo) of GF(4)
    def g16_add(self, a, b):
        return (self.g4_add(a[0], b[0]), self.g4_add(a[1], b[1]))

    def g16_sq(self, a):                      # a1^2 y + (a1^2 nu + a0^2)
        s1 = self.g4_sq(a[0])
        return (s1, self.g4_add(self.g4_scale(s1, self.nu), self.g4_sq(a[1])))

    def g16_scale(self, a, c):
        c1, c0 = c >> 2, c & 3
        t11 = self.g4_scale(a[0], c1)
        hi = self.g4_add(self.g4_add(self.g4_scale(a[0], c0), self.g4_scale(a[1], c1)), t11)
        lo = self.g4_add(self.g4_scale(t11, self.nu), self.g4_scale(a[1], c0))
        return (hi, lo)

    def g16_mul(self, a, b):
        p11 = self.g4_mul(a[0], b[0])
        p00 = self.g4_mul(a[1], b[1])
        pss = self.g4_mul(self.g4_add(a[0], a[1]), self.g4_add(b[0], b[1]))
        return (self.g4_add(pss, p00), self.g4_add(self.g4_scale(p11, self.nu), p00))

    def g16_inv(self, d):
        e = self.g4_add(self.g4_add(self.g4_scale(self.g4_sq(d[0]), self.nu), self.g4_mul(d[0], d[1])),
                        self.g4_sq(d[1]))
        einv = self.g4_sq(e)                  # in GF(4) the inverse is the square (0 -> 0)
        return (self.g4_mul(d[0], einv), self.g4_mul(self.g4_add(d[0], d[1]), einv))

    def g256_inv(self, a):
        a1, a0 = a
        d = self.g16_add(self.g16_add(self.g16_scale(self.g16_sq(a1), self.lam), self.g16_mul(a1, a0)),
                         self.g16_sq(a0))
        dinv = self.g16_inv(d)
        return (self.g16_mul(a1, dinv), self.g16_mul(self.g16_add(a1, a0), dinv))


def flatten256(v):
    """Tower element (GF16 hi, GF16 lo) -> 8 linear forms, bit i of the int code."""
    (h1, h0), (l1, l0) = v
    # int code: (hi16 << 4) | lo16, hi16 = (h1 << 2) | h0, each GF(4) = (b1 << 1) | b0
    return [l0[1], l0[0], l1[1], l1[0], h0[1], h0[0], h1[1], h1[0]]


def unflatten256(bits):
    return (((bits[7], bits[6]), (bits[5], bits[4])), ((bits[3], bits[2]), (bits[1], bits[0])))


# ---------------------------------------------------------------- XOR network

def xor_network(targets, order_key):
    """Paar's greedy heuristic: targets is a list of frozensets of signals;
    returns (list of (name, a, b) XOR nodes, list of target signal names)."""
    rows = [set(t) for t in targets]
    nodes = []
    k = 0
    while True:
        counts = {}
        for r in rows:
            if len(r) < 2:
                continue
            for pair in itertools.combinations(sorted(r, key=order_key), 2):
                counts[pair] = counts.get(pair, 0) + 1
        if not counts:
            break
        best = max(counts.items(), key=lambda kv: (kv[1], [-order_key(s) for s in kv[0]]))[0]
        name = f"n{k}"
        k += 1
        nodes.append((name, best[0], best[1]))
        for r in rows:
            if best[0] in r and best[1] in r:
                r.discard(best[0])
                r.discard(best[1])
                r.add(name)
    outs = []
    for r in rows:
        outs.append(next(iter(r)) if r else None)
    return nodes, outs


def build(nu, lam, beta, powers):
    m = mat_from_columns(powers)            # AES basis -> tower basis
    minv = mat_inverse(m)
    # AES affine matrix, rows as masks over the inverse's bits
    a = [(1 << i) | (1 << ((i + 4) % 8)) | (1 << ((i + 5) % 8)) | (1 << ((i + 6) % 8)) | (1 << ((i + 7) % 8))
         for i in range(8)]
    out_map = [0] * 8                        # rows of A * M^-1 over tower bits
    for i in range(8):
        for j in range(8):
            if (a[i] >> j) & 1:
                out_map[i] ^= minv[j]
    core = Core(nu, lam)
    x = [frozenset([f"x{i}"]) for i in range(8)]
    t = []
    for i in range(8):
        f = frozenset()
        for j in range(8):
            if (m[i] >> j) & 1:
                f = f ^ x[j]
        t.append(f)
    u = flatten256(core.g256_inv(unflatten256(t)))
    s = []
    for i in range(8):
        f = frozenset()
        for j in range(8):
            if (out_map[i] >> j) & 1:
                f = f ^ u[j]
        s.append(f)
    return core.ands, s


def order_key_factory(ands):
    idx = {name: i for i, (name, _, _) in enumerate(ands)}

    def key(sig):
        if sig.startswith("x"):
            return -1000 + int(sig[1:])
        if sig.startswith("g"):
            return idx[sig]
        return 10 ** 6 + int(sig[1:])
    return key


def compile_circuit(ands, outs):
    """Straight-line program: list of (name, op, args) in dependency order."""
    targets = []
    for _, la, lb in ands:
        targets += [la, lb]
    targets += outs
    key = order_key_factory(ands)
    nodes, names = xor_network(targets, key)
    defs = {n: ("xor", a, b) for n, a, b in nodes}
    for i, (g, _, _) in enumerate(ands):
        defs[g] = ("and", names[2 * i], names[2 * i + 1])
    out_names = names[2 * len(ands):]
    prog, done = [], set(f"x{i}" for i in range(8))

    def emit(sig):
        if sig is None or sig in done:
            return
        op, a, b = defs[sig]
        emit(a)
        emit(b)
        prog.append((sig, op, a, b))
        done.add(sig)
    for o in out_names:
        emit(o)
    return prog, out_names


def evaluate(prog, out_names, const, v):
    """Bit-level evaluation of the program on 256-lane integers (lane = input)."""
    env = {f"x{i}": v[i] for i in range(8)}
    full = (1 << 256) - 1
    for name, op, a, b in prog:
        env[name] = env[a] & env[b] if op == "and" else env[a] ^ env[b]
    res = []
    for i, o in enumerate(out_names):
        w = env[o] if o is not None else 0
        if (const >> i) & 1:
            w ^= full
        res.append(w)
    return res


def check(prog, out_names):
    sbox = aes_sbox()
    v = [sum(((a >> i) & 1) << a for a in range(256)) for i in range(8)]
    r = evaluate(prog, out_names, 0x63, v)
    got = [sum(((r[i] >> a) & 1) << i for i in range(8)) for a in range(256)]
    return got == sbox


def best_circuit():
    best = None
    for nu, lam, beta, powers in tower_choices():
        ands, outs = build(nu, lam, beta, powers)
        prog, out_names = compile_circuit(ands, outs)
        cost = len(prog)
        if best is None or cost < best[0]:
            best = (cost, nu, lam, beta, prog, out_names)
    return best


def render(best):
    cost, nu, lam, beta, prog, out_names = best
    n_and = sum(1 for p in prog if p[1] == "and")
    lines = [
        "// GENERATED by gen_sbox_circuit.py -- do not edit.",
        "// The AES S-box (FIPS-197 section 5.1.1) as a straight-line circuit on",
        "// 32-bit words: bit k of x_i is bit i of the k-th of 32 independent inputs.",
        f"// Composite field GF(((2^2)^2)^2): nu = {nu}, lambda = {lam}, beta = 0x{beta:02x};",
        f"// {n_and} AND + {cost - n_and} XOR gates, plus NOTs for the affine constant 0x63",
        "// (the compiler merges them into three-input LOP3 operations).",
        "#pragma once",
        "#include <cstdint>",
        "",
        "namespace kgpu {",
        "",
        "__device__ __forceinline__ void sbox_circuit(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,",
        "                                             uint32_t& x4, uint32_t& x5, uint32_t& x6, uint32_t& x7) {",
    ]
    for name, op, a, b in prog:
        sym = "&" if op == "and" else "^"
        lines.append(f"    const uint32_t {name} = {a} {sym} {b};")
    for i, o in enumerate(out_names):
        val = o if o is not None else "0u"
        if (0x63 >> i) & 1:
            val = f"~{val}"
        lines.append(f"    x{i} = {val};")
    lines += ["}", "", "}  // namespace kgpu", ""]
    return "\n".join(lines)


def main():
    best = best_circuit()
    if not check(best[4], best[5]):
        sys.exit("generated circuit does not match the S-box")
    text = render(best)
    if "--check" in sys.argv:
        with open(OUT) as f:
            sys.exit(0 if f.read() == text else 1)
    with open(OUT, "w") as f:
        f.write(text)
    n_and = sum(1 for p in best[4] if p[1] == "and")
    print(f"nu={best[1]} lam={best[2]} beta=0x{best[3]:02x}: {n_and} AND + {best[0] - n_and} XOR -> {OUT}")


if __name__ == "__main__":
    main()
