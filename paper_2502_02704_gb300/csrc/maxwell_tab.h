// Float32 Maxwellian factor tables of the storage form (fine.cu), evaluated
// to within about 1e-9 relative before the single rounding to float32, with
// float32 arithmetic only.
//
// Why: an entry exp(-(v_j - u)^2 / (2 theta)) whose exponent is formed in
// float32 from float32 copies of v_j, u and 1/(2 theta) carries an error of
// about x * 1e-7 relative (x the exponent), and the same entry feeds nv^2
// cells, so the error does not average out of the moments: it was the
// largest part of the mixed-precision scheme's moment error.  Here the
// parameters arrive as float pairs (hi + lo, about 48 bits) from the float64
// Maxwellian parameters, the exponent is formed in pair arithmetic on the
// grid coordinate k_j = (v_j + L)/dv - 1/2 - (nv - 1)/2, which is an exact
// half-integer, and exp is evaluated by the textbook method of Cody and
// Waite (argument reduction by a two-part ln 2, then the Taylor series of
// exp on |r| <= ln2/2 with its first terms in pair arithmetic).  This keeps
// the whole table on the float32 pipes; this part's float64 pipe is ~1/64
// of their rate and the tables sit on the critical path between two steps.
#pragma once
#include <math.h>

namespace prk {

// Per-cell table parameters: (u_d / dv) for d = x, y, z, w = dv^2 / (2 theta)
// and the prefactor weight rho (2 pi theta)^{-3/2}, each as a float pair.
struct TabPar {
    float uh[3], ul[3];
    float wh, wl;
    float ph, pl;
};

__host__ __device__ __forceinline__ void split_pair(double x, float& h, float& l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

// From the float64 parameters u (3), theta and the prefactor (weight included).
__host__ __device__ __forceinline__ TabPar make_tabpar(const double* u, double theta, double pref, double dv)
{
    TabPar P;
    const double idv = 1.0 / dv;
    for (int d = 0; d < 3; ++d) split_pair(u[d] * idv, P.uh[d], P.ul[d]);
    split_pair(dv * dv / (2.0 * theta), P.wh, P.wl);
    split_pair(pref, P.ph, P.pl);
    return P;
}

// Grid coordinate of node j: v_j / dv = j + 1/2 - nv/2 (exact in float32).
__host__ __device__ __forceinline__ float node_k(int j, int nv) { return (float)j + 0.5f - 0.5f * (float)nv; }

// s + e = a + b exactly (Knuth's two-sum).
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Float pairs h + l (|l| <= ulp(h)/2 after normalisation, ~48 bits): the
// table weights 3/(2 tau) and rho (2 pi theta)^{-3/2} are formed in pair
// arithmetic from the float64 Maxwellian parameters, so that no float64
// division or square root (tens of instructions on this part's narrow
// float64 pipe) sits between two steps.  Products with Dekker's method
// (exact float products by FMA), reciprocal and square root by one Newton
// step from the float32 value; relative error ~1e-13.
struct F2 {
    float h, l;
};

__host__ __device__ __forceinline__ F2 f2_of(double x)
{
    F2 r;
    split_pair(x, r.h, r.l);
    return r;
}
__host__ __device__ __forceinline__ F2 f2_norm(float h, float e)
{
    const float s = h + e;
    return F2{s, e - (s - h)};
}
__host__ __device__ __forceinline__ F2 f2_mul(F2 a, F2 b)
{
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p) + fmaf(a.h, b.l, a.l * b.h);
    return f2_norm(p, e);
}
// 1 / a: r = 1/a_h, then r + r (1 - a r) with the residual in pair arithmetic
__host__ __device__ __forceinline__ F2 f2_rcp(F2 a)
{
    const float r = 1.0f / a.h;
    const float t = fmaf(-a.h, r, 1.0f) - a.l * r;
    return f2_norm(r, r * t);
}
// sqrt(a): s = sqrt(a_h), then s + (a - s^2) / (2 s)
__host__ __device__ __forceinline__ F2 f2_sqrt(F2 a)
{
    const float s = sqrtf(a.h);
    const float d = fmaf(-s, s, a.h) + a.l;
    return f2_norm(s, d * (0.5f / s));
}

// exp(-(xh + xl)) for xh >= 0 to about 1e-9 relative, times the pair
// (mh + ml), rounded once to float32.  Cody-Waite: -x = n ln2 + r with n an
// integer and |r| <= ln2/2; ln2 = LN2H + LN2L with LN2H holding 15
// significant bits, so n * LN2H is exact and rh = -xh - n LN2H is exact
// (Sterbenz).  exp(r) = 1 + r + r^2/2 + r^3 S(r): the leading three terms in
// pair arithmetic, S(r) = 1/6 + r/24 + ... + r^6/362880 (Taylor, truncation
// below 1e-11 on the interval) in float32; exp(rl) = 1 + rl + rl^2/2 for the
// low part (|rl| <= ~2e-4: the next term is below 1e-11).
__host__ __device__ __forceinline__ float exp_neg_pair(float xh, float xl, float mh, float ml)
{
    if (!(xh < 103.0f)) return 0.0f;  // below the float32 range (also catches NaN arguments)
    const float LOG2E = 1.44269504088896341f;
    const float LN2H = 0.693145751953125f;       // 22713 / 32768
    const float LN2L = 1.428606820309417232e-6f;  // ln 2 - LN2H
    const float n = rintf(-xh * LOG2E);
    const float rh = fmaf(-n, LN2H, -xh);
    const float rl = fmaf(-n, LN2L, -xl);
    float p = 1.0f / 362880.0f;
    p = fmaf(p, rh, 1.0f / 40320.0f);
    p = fmaf(p, rh, 1.0f / 5040.0f);
    p = fmaf(p, rh, 1.0f / 720.0f);
    p = fmaf(p, rh, 1.0f / 120.0f);
    p = fmaf(p, rh, 1.0f / 24.0f);
    p = fmaf(p, rh, 1.0f / 6.0f);
    const float r2 = rh * rh;
    const float qh = 0.5f * r2, ql = 0.5f * fmaf(rh, rh, -r2);
    float s1, e1, s2, e2;
    two_sum(1.0f, rh, s1, e1);
    two_sum(s1, qh, s2, e2);
    float lo = e1 + e2 + ql + r2 * rh * p;
    lo = fmaf(s2 + lo, fmaf(0.5f * rl, rl, rl), lo);  // times exp(rl) = 1 + rl + rl^2 / 2
    // (s2 + lo) (mh + ml), one rounding
    const float hi = s2 * mh;
    const float err = fmaf(s2, mh, -hi) + fmaf(lo, mh, s2 * ml);
    return ldexpf(hi + err, (int)n);
}

// Table entry of dimension d at node j: exp(-(k_j - u_d/dv)^2 w), times the
// prefactor for d = 0 (T0 carries weight rho (2 pi theta)^{-3/2}).
__host__ __device__ __forceinline__ float tab_entry(const TabPar& P, int d, float kj)
{
    float ch, cl;
    two_sum(kj, -P.uh[d], ch, cl);
    cl -= P.ul[d];
    const float sh = ch * ch;
    const float sl = fmaf(ch, ch, -sh) + 2.0f * ch * cl;
    const float xh = sh * P.wh;
    const float xl = fmaf(sh, P.wh, -xh) + fmaf(sh, P.wl, sl * P.wh);
    return d == 0 ? exp_neg_pair(xh, xl, P.ph, P.pl) : exp_neg_pair(xh, xl, 1.0f, 0.0f);
}

}  // namespace prk
