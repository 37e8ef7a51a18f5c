"""Generate ``codelets.cuh``: straight-line in-register DFTs of small sizes.

Each codelet computes X[k] = sum_n x[n] exp(s*2*pi*i*n*k/R) in place on an
array of R complex values held in registers (s = -1 forward, +1 inverse,
unnormalised).  Sizes are built by recursive decimation in time from radix-2,
-3 and -4 butterflies and, for other prime factors p, a direct length-p DFT
that pairs inputs n and p - n (their sum meets the cosines, their difference
the sines); twiddles that are powers of i cost nothing, odd multiples of pi/4
cost two multiplies, the rest are complex multiplies by literal constants.
Run:  python gen_codelets.py > codelets.cuh
"""
import math
import sys

SIZES = (2, 3, 4, 5, 6, 8, 12, 13, 16, 20, 24, 26, 32)

# Two-step plans N = R1 * R2 of the strided passes (must match Plan<N> in
# psc_common.cuh).  An inverse pass zero-pads its lines from 2K+1 to N points
# (K = (N-1)//3), so inputs n1 of its first DFT (positions R2 n1 + n2) are zero
# for every n2 when R2 n1 > K and R2 n1 + R2 - 1 < N - K: those DFTs are also
# generated with that input range known to be zero.
PLANS = {8: (4, 2), 12: (4, 3), 16: (4, 4), 24: (6, 4), 32: (8, 4), 48: (12, 4), 64: (8, 8),
         96: (12, 8), 128: (16, 8), 192: (24, 8), 256: (16, 16), 512: (32, 16), 520: (20, 26),
         1024: (32, 32)}


def zero_range(N):
    R1, R2 = PLANS[N]
    K = (N - 1) // 3
    zs = [n1 for n1 in range(R1) if R2 * n1 > K and R2 * n1 + R2 - 1 < N - K]
    return (R1, zs[0], zs[-1]) if zs else None


class Emitter:
    """Emits straight-line code; a value None is a known zero, which the
    operations propagate instead of computing."""

    def __init__(self):
        self.lines = []
        self.n = 0

    def new(self, re, im):
        v = f"v{self.n}"
        self.n += 1
        self.lines.append(f"    const T {v}r = {re}, {v}i = {im};")
        return (v + "r", v + "i")

    def add(self, a, b):
        if a is None:
            return b
        if b is None:
            return a
        return self.new(f"{a[0]} + {b[0]}", f"{a[1]} + {b[1]}")

    def sub(self, a, b):
        if b is None:
            return a
        if a is None:
            return self.new(f"-{b[0]}", f"-{b[1]}")
        return self.new(f"{a[0]} - {b[0]}", f"{a[1]} - {b[1]}")

    def rot(self, a, q):
        """a * i^q without arithmetic (negations fold into later adds)."""
        if a is None:
            return None
        q %= 4
        if q == 0:
            return a
        if q == 1:
            return self.new(f"-{a[1]}", f"{a[0]}")
        if q == 2:
            return self.new(f"-{a[0]}", f"-{a[1]}")
        return self.new(f"{a[1]}", f"-{a[0]}")

    def twiddle(self, a, m, R, s):
        """a * exp(s*2*pi*i*m/R)."""
        if a is None:
            return None
        m %= R
        if m == 0:
            return a
        if (4 * m) % R == 0:
            return self.rot(a, s * (4 * m) // R)
        if (8 * m) % R == 0:
            # exp(i*pi*(2q+1)/4) = (c + i c') with |c| = |c'| = sqrt(1/2)
            q = ((s * (8 * m) // R) % 8 - 1) // 2
            b = self.new(f"T(0.70710678118654752) * ({a[0]} - {a[1]})",
                         f"T(0.70710678118654752) * ({a[0]} + {a[1]})")
            return self.rot(b, q)
        th = s * 2.0 * math.pi * m / R
        c, sn = math.cos(th), math.sin(th)
        return self.new(f"{a[0]} * T({c!r}) - {a[1]} * T({sn!r})",
                        f"{a[0]} * T({sn!r}) + {a[1]} * T({c!r})")

    def dft(self, xs, s):
        R = len(xs)
        if R == 1:
            return list(xs)
        if R == 2:
            return [self.add(xs[0], xs[1]), self.sub(xs[0], xs[1])]
        if R == 3:
            a, b, c = xs
            t1 = self.add(b, c)
            if t1 is None:
                t2 = a
            elif a is None:
                t2 = self.new(f"-T(0.5) * {t1[0]}", f"-T(0.5) * {t1[1]}")
            else:
                t2 = self.new(f"{a[0]} - T(0.5) * {t1[0]}", f"{a[1]} - T(0.5) * {t1[1]}")
            h = 0.86602540378443865 * s  # s * sqrt(3)/2
            d = self.sub(b, c)
            t3 = None if d is None else self.new(f"-T({h!r}) * {d[1]}", f"T({h!r}) * {d[0]}")
            return [self.add(a, t1), self.add(t2, t3), self.sub(t2, t3)]
        if R == 4:
            a, b, c, d = xs
            t0, t1 = self.add(a, c), self.sub(a, c)
            t2 = self.add(b, d)
            t3 = self.rot(self.sub(b, d), s)
            return [self.add(t0, t2), self.add(t1, t3), self.sub(t0, t2), self.sub(t1, t3)]
        P = 4 if R % 4 == 0 else (2 if R % 2 == 0 else (3 if R % 3 == 0 else smallest_factor(R)))
        if P == R:
            return self.prime_dft(xs, s)
        Q = R // P
        Y = {}
        for n2 in range(Q):
            y = self.dft([xs[Q * n1 + n2] for n1 in range(P)], s)
            for k1 in range(P):
                Y[n2, k1] = self.twiddle(y[k1], n2 * k1, R, s)
        X = [None] * R
        for k1 in range(P):
            z = self.dft([Y[n2, k1] for n2 in range(Q)], s)
            for k2 in range(Q):
                X[k1 + P * k2] = z[k2]
        return X


    def lincomb(self, terms):
        """sum of coef * value over (coef, value) pairs with known-zero values
        dropped; a string, or None if every value is zero."""
        parts = [f"{v} * T({c!r})" if c != 1.0 else v for c, v in terms if v is not None]
        return " + ".join(parts) if parts else None

    def prime_dft(self, xs, s):
        """Direct DFT of odd prime length R: with a_j = x_j + x_{R-j} and
        b_j = x_j - x_{R-j} (j = 1 .. (R-1)/2),
        X_k = x_0 + sum_j cos(2 pi j k/R) a_j + i s sum_j sin(2 pi j k/R) b_j and
        X_{R-k} the same with the sine sum negated."""
        R = len(xs)
        h = (R - 1) // 2
        a = [None] + [self.add(xs[j], xs[R - j]) for j in range(1, h + 1)]
        b = [None] + [self.sub(xs[j], xs[R - j]) for j in range(1, h + 1)]
        X = [None] * R
        x0 = xs[0]
        X[0] = x0
        for j in range(1, h + 1):
            X[0] = self.add(X[0], a[j])
        for k in range(1, h + 1):
            c = [math.cos(2.0 * math.pi * j * k / R) for j in range(h + 1)]
            sn = [s * math.sin(2.0 * math.pi * j * k / R) for j in range(h + 1)]
            ar = self.lincomb([(1.0, None if x0 is None else x0[0])] +
                              [(c[j], None if a[j] is None else a[j][0]) for j in range(1, h + 1)])
            ai = self.lincomb([(1.0, None if x0 is None else x0[1])] +
                              [(c[j], None if a[j] is None else a[j][1]) for j in range(1, h + 1)])
            br = self.lincomb([(sn[j], None if b[j] is None else b[j][0]) for j in range(1, h + 1)])
            bi = self.lincomb([(sn[j], None if b[j] is None else b[j][1]) for j in range(1, h + 1)])
            A = None if ar is None else self.new(ar, ai)
            Bv = None if br is None else self.new(br, bi)
            iB = self.rot(Bv, 1)
            X[k] = self.add(A, iB)
            X[R - k] = self.sub(A, iB)
        return X


def smallest_factor(R):
    f = 2
    while R % f:
        f += 1
    return f


def codelet(R, s, zero=None):
    """zero = (z0, z1): inputs z0..z1 are known to be zero and are not read."""
    e = Emitter()
    xs = []
    for i in range(R):
        if zero and zero[0] <= i <= zero[1]:
            xs.append(None)
            continue
        e.lines.append(f"    const T in{i}r = x[{i}].x, in{i}i = x[{i}].y;")
        xs.append((f"in{i}r", f"in{i}i"))
    X = e.dft(xs, s)
    for k in range(R):
        if X[k] is None:
            e.lines.append(f"    x[{k}].x = T(0); x[{k}].y = T(0);")
        else:
            e.lines.append(f"    x[{k}].x = {X[k][0]}; x[{k}].y = {X[k][1]};")
    name = "fwd" if s < 0 else "inv"
    body = "\n".join(e.lines)
    if zero:
        head = f"template <> struct DftZ<{R}, {s}, {zero[0]}, {zero[1]}> {{\n"
        name += f" {R}, inputs {zero[0]}..{zero[1]} zero"
    else:
        head = f"template <> struct Dft<{R}, {s}> {{\n"
        name += f" {R}"
    return (head + f"  template <typename T, typename C>\n"
            f"  static __device__ __forceinline__ void run(C* x) {{  // {name}\n{body}\n  }}\n}};\n")


def main(out=sys.stdout):
    out.write("// Generated by gen_codelets.py -- do not edit.\n")
    out.write("// In-place, in-register DFTs: X[k] = sum_n x[n] exp(s 2 pi i n k / R).\n")
    out.write("#pragma once\n\nnamespace psc {\n\n")
    out.write("template <int R, int S> struct Dft;\n")
    out.write("// inputs Z0..Z1 known to be zero\n")
    out.write("template <int R, int S, int Z0, int Z1> struct DftZ;\n\n")
    for R in SIZES:
        for s in (-1, 1):
            out.write(codelet(R, s))
            out.write("\n")
    done = set()
    for N in sorted(PLANS):
        z = zero_range(N)
        if z and z not in done:
            done.add(z)
            out.write(codelet(z[0], 1, (z[1], z[2])))
            out.write("\n")
    out.write("}  // namespace psc\n")


if __name__ == "__main__":
    main()
