"""Pure (real solid-harmonic) shells: the Cartesian-to-pure coefficient table.

The ERI kernels work on Cartesian components (Sec. 2.2, Eq. 1).  A pure d or f
shell is a fixed combination of them: column m of T_l holds the coefficients
of the real solid harmonic S_lm on the library's normalised Cartesian
components (lx descending, then ly descending), for m = -l, ..., l.  The
closed form is the triple sum of Helgaker, Jorgensen & Olsen, Molecular
Electronic-Structure Theory (2000), Eqs. 6.4.47-6.4.50:

    S_lm = N_lm sum_{t=0}^{floor((l-|m|)/2)} sum_{u=0}^{t} sum_{v}
           (-1)^(t+v-v_m) (1/4)^t C(l,t) C(l-t,|m|+t) C(t,u) C(|m|,2v)
           x^(2t+|m|-2(u+v)) y^(2(u+v)) z^(l-2t-|m|),
    N_lm = sqrt(2 (l+|m|)! (l-|m|)! / 2^delta_m0) / (2^|m| l!),

with v_m = 0 (m >= 0) or 1/2 (m < 0) and v = v_m, v_m+1, ..., up to
floor(|m|/2 - v_m) + v_m.  With this N_lm every S_lm has the norm of the
axial component x^l, which is the norm the library gives a contracted
Cartesian shell, so the coefficients apply to normalised components as they
stand.  s and p shells are not transformed (T_0 = 1, T_1 = I_3).

The table is emitted as a C array (``sph_table.cu``) that the runtime uploads
for the transform kernel in ``csrc/sph_transform.cuh``.
"""
from __future__ import annotations

import math
import os

LMAX = 3


def cart_components(l):
    return [(lx, l - lx - lz, lz) for lx in range(l, -1, -1) for lz in range(0, l - lx + 1)]


def npure(l):
    return 2 * l + 1 if l >= 2 else (l + 1) * (l + 2) // 2


def solid_harmonic(l, m):
    """{(a, b, c): coefficient} of S_lm (closed form above)."""
    am = abs(m)
    twice_vm = 0 if m >= 0 else 1                       # 2 v_m
    norm = math.sqrt(2.0 * math.factorial(l + am) * math.factorial(l - am) / (2.0 if m == 0 else 1.0)) \
        / (2 ** am * math.factorial(l))
    poly = {}
    for t in range((l - am) // 2 + 1):
        for u in range(t + 1):
            # v runs over v_m + k, k = 0 .. floor(|m|/2 - v_m); kept in units of 1/2
            kmax = (am - twice_vm) // 2
            for k in range(kmax + 1):
                twice_v = twice_vm + 2 * k
                c = (-1) ** (t + k) * 0.25 ** t * math.comb(l, t) * math.comb(l - t, am + t) \
                    * math.comb(t, u) * math.comb(am, twice_v)
                e = (2 * t + am - 2 * u - twice_v, 2 * u + twice_v, l - 2 * t - am)
                poly[e] = poly.get(e, 0.0) + norm * c
    return {e: c for e, c in poly.items() if c != 0.0}


def table(l):
    """T_l as a list of ncart(l) rows of npure(l) coefficients."""
    comps = cart_components(l)
    if l <= 1:
        return [[1.0 if i == j else 0.0 for j in range(len(comps))] for i in range(len(comps))]
    T = [[0.0] * (2 * l + 1) for _ in comps]
    for col, m in enumerate(range(-l, l + 1)):
        for e, c in solid_harmonic(l, m).items():
            T[comps.index(e)][col] = c
    return T


def offsets(lmax=LMAX):
    off = [0]
    for l in range(lmax + 1):
        off.append(off[-1] + len(cart_components(l)) * npure(l))
    return off


def emit(outdir, lmax=LMAX):
    """Write sph_table.cu: the concatenated row-major tables and their offsets."""
    vals = [c for l in range(lmax + 1) for row in table(l) for c in row]
    off = offsets(lmax)
    body = ",\n  ".join(", ".join(repr(v) for v in vals[i:i + 6]) for i in range(0, len(vals), 6))
    text = f"""// Generated by codegen/sph_codegen.py: Cartesian-to-pure coefficient tables,
// per l = 0..{lmax} an ncart(l) x npure(l) row-major block starting at k_sph_off[l].
static const double k_sph_coef[{len(vals)}] = {{
  {body}
}};
static const int k_sph_off[{lmax + 2}] = {{{", ".join(map(str, off))}}};
// Returns the highest l tabulated; *coef and *off point at static host arrays.
extern "C" int gb_sph_table(const double** coef, const int** off) {{
  *coef = k_sph_coef;
  *off = k_sph_off;
  return {lmax};
}}
"""
    fn = os.path.join(outdir, "sph_table.cu")
    if not (os.path.exists(fn) and open(fn).read() == text):
        with open(fn, "w") as f:
            f.write(text)
    return fn
