// Closed form of the integral of S2 over the truncated mesh rectangle
// (Eq. IS2, "exactly in terms of logarithms"), written with asinh.
#pragma once
#include <math.h>

// G(s, t) with d^2 G / ds dt = (A s^2 + B s t + C t^2)^(-1/2), D = 4AC - B^2 > 0:
//   s / sqrt(C) asinh((B s + 2 C t) / (sqrt(D) |s|)) + t / sqrt(A) asinh((2 A s + B t) / (sqrt(D) |t|)),
// each term taken as its limit 0 where its prefactor vanishes.  (The
// logarithmic antiderivative ln(2 sqrt(A Q) + 2 A s + B t) differs from the
// asinh form by functions of one variable, which cancel in a rectangle.)
__device__ __forceinline__ double swj_G_corner(double A, double B, double C, double sD,
                                               double rsA, double rsC, double s, double t)
{
    double v = 0.0;
    if (s != 0.0) v += s * rsC * asinh((B * s + 2.0 * C * t) / (sD * fabs(s)));
    if (t != 0.0) v += t * rsA * asinh((2.0 * A * s + B * t) / (sD * fabs(t)));
    return v;
}

// int_{s1}^{s2} int_{t1}^{t2} (A s^2 + B s t + C t^2)^(-1/2) dt ds
__device__ __forceinline__ double swj_rect_int(double A, double B, double C, double s1,
                                               double s2, double t1, double t2)
{
    double sD = sqrt(4.0 * A * C - B * B);
    double rsA = 1.0 / sqrt(A), rsC = 1.0 / sqrt(C);
    return swj_G_corner(A, B, C, sD, rsA, rsC, s2, t2) - swj_G_corner(A, B, C, sD, rsA, rsC, s1, t2)
         - swj_G_corner(A, B, C, sD, rsA, rsC, s2, t1) + swj_G_corner(A, B, C, sD, rsA, rsC, s1, t1);
}

// I of Eq. IS2 for the target (k + 1/2, l) (0-based k, l) of an N x M mesh:
// the direct part over [x1 - x*, xN - x*] x [-y*, yM - y*] plus the image
// part (B -> -B, t = y + y*) over [.., ..] x [y*, yM + y*].
__device__ __forceinline__ double swj_I_S2(double A, double B, double C, int N, int M, int k,
                                           int l, double dx, double dy)
{
    double s1 = -((double)k + 0.5) * dx;
    double s2 = ((double)(N - 1 - k) - 0.5) * dx;
    double yt = (double)l * dy;
    double yM = (double)(M - 1) * dy;
    return swj_rect_int(A, B, C, s1, s2, -yt, yM - yt) + swj_rect_int(A, -B, C, s1, s2, yt, yM + yt);
}
