"""Floating-point parity bar shared by the GPU tests.

The bar is 1e-10 relative (|got - ref| / |ref|) against the oracle.  It is
held wherever a correct FP64 evaluation of the sum can meet it: a sum whose
terms carry FP64 rounding (about n units of 2^-53 each) errs by at most about
n 2^-53 kappa relative, kappa = sum|t| / |per| the condition number of the
sum; with a safety factor of 4 the bar applies whenever
4 n 2^-53 kappa <= 1e-10 (kappa up to about 5.6e3 at n = 40).  Beyond that
(the closed forms J_n, J - I and other sums with extreme cancellation, whose
permanents are tiny against their terms) no FP64 algorithm reaches 1e-10,
and the a-posteriori bound 64 n u sum|t| of the arithmetic in use (u = 2^-53
for FP64 products, 2^-46 for double-float ones) applies instead.  Every check
prints the observed error, kappa and which bound applied.
"""
from __future__ import annotations

REL = 1e-10
U64 = 2.0 ** -53
U_DF = 2.0 ** -46


def unit(rows: str) -> float:
    """Unit roundoff of a row/product arithmetic (PERM_ROWS value)."""
    return U_DF if rows in ("pdf", "df", "pair") else U64


def bar_reachable(n: int, kappa: float) -> bool:
    return 4.0 * n * U64 * kappa <= REL


def check(got, ref, asum: float, n: int, u: float = U64, what: str = "") -> float:
    """Assert the parity bar for one result; returns the relative error."""
    err = abs(got - ref)
    if ref == 0:
        print(f"{what}: |err| {err:.3e} (exact zero reference), bound 64 n u sum|t|")
        assert err <= 64 * n * u * asum, (what, got, ref, asum)
        return err
    rel = err / abs(ref)
    kappa = asum / abs(ref)
    if bar_reachable(n, kappa):
        print(f"{what}: rel err {rel:.3e}, kappa {kappa:.3e}, bound 1e-10 relative")
        assert rel <= REL, (what, got, ref, rel, kappa)
    else:
        bound = 64 * n * u * asum
        print(f"{what}: rel err {rel:.3e}, kappa {kappa:.3e} (1e-10 out of reach for FP64), "
              f"bound 64 n u sum|t| = {bound / abs(ref):.3e} relative")
        assert err <= bound, (what, got, ref, rel, kappa)
    return rel
