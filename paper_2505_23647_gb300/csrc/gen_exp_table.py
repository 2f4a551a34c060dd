"""Print the constants of expcr.cuh: for the quick phase of exp_cr the table
2^(j/64), j = 0..63, as double-double pairs (hi = RN(2^(j/64)),
lo = RN(2^(j/64) - hi)), and ln2/64 split for a Cody-Waite reduction (C1
with 32 significant bits, so that k C1 is exact for |k| < 2^21; C2 =
RN(ln2/64 - C1)), and RN(64/ln2); for log_dd the reciprocals 1/(2j+1),
j = 0..20, as double-double pairs; for the quick phase of pow_cr 1/F and
ln F, F = 1 + j/128, j = 0..128, as double-double pairs.  Evaluated with 80 significant digits
(mpmath).  Run: python gen_exp_table.py > table.txt and paste."""
import mpmath

mpmath.mp.dps = 80


def rn(v):
    """Nearest binary64 to the mpmath value v (mpmath rounds to nearest)."""
    return float(mpmath.mpf(v))


def main():
    rows = []
    for j in range(64):
        t = mpmath.power(2, mpmath.mpf(j) / 64)
        hi = rn(t)
        lo = rn(t - mpmath.mpf(hi))
        rows.append(f"    {{{float.hex(hi)}, {float.hex(lo)}}},   // 2^({j}/64)")
    print("\n".join(rows))
    l = mpmath.log(2) / 64
    e = int(mpmath.floor(mpmath.log(l, 2)))          # l in [2^e, 2^(e+1))
    scale = mpmath.mpf(2) ** (31 - e)                  # 32 significant bits
    c1 = mpmath.floor(l * scale) / scale
    c2 = rn(l - c1)
    print(f"C1 = {float.hex(rn(c1))}")
    print(f"C2 = {float.hex(c2)}")
    print(f"INV = {float.hex(rn(64 / mpmath.log(2)))}")
    # the reciprocals 1/(2j+1) of log_dd's atanh series: hi = RN(1/d),
    # lo = RN((1 - hi d)/d) (the exact residual rounded once)
    for j in range(21):
        d = 2 * j + 1
        hi = rn(mpmath.mpf(1) / d)
        lo = rn((1 - mpmath.mpf(hi) * d) / d)
        print(f"    {{{float.hex(hi)}, {float.hex(lo)}}},   // 1/{d}")
    # the quick phase of pow_cr: F_j = 1 + j/128, j = 0..128, with 1/F_j and
    # ln F_j as double-double pairs
    for j in range(129):
        F = 1 + mpmath.mpf(j) / 128
        ih = rn(1 / F)
        il = rn(1 / F - mpmath.mpf(ih))
        lh = rn(mpmath.log(F))
        ll = rn(mpmath.log(F) - mpmath.mpf(lh))
        print(f"    {{{float.hex(ih)}, {float.hex(il)}, {float.hex(lh)}, {float.hex(ll)}}},   // F = 1 + {j}/128")


if __name__ == "__main__":
    main()
