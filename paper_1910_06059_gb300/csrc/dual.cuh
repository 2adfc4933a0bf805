// Forward-mode dual numbers for the device (Section 2.4 of arXiv 1910.06059:
// a value carried with its first derivatives, products by the product rule).
// D3 carries the derivatives with respect to one cell's three primary
// variables (p_o, s_w, x).  Face quantities seed the two cells separately,
// so their derivatives stay two D3-sized halves instead of a dense 6-vector.
#pragma once

namespace bo {

struct D3 {
    double v, d0, d1, d2;
};

__device__ __forceinline__ D3 dconst(double c) { return {c, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ D3 dvar(double v, int slot) {
    return {v, slot == 0 ? 1.0 : 0.0, slot == 1 ? 1.0 : 0.0, slot == 2 ? 1.0 : 0.0};
}
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return {a.v + b.v, a.d0 + b.d0, a.d1 + b.d1, a.d2 + b.d2}; }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return {a.v - b.v, a.d0 - b.d0, a.d1 - b.d1, a.d2 - b.d2}; }
__device__ __forceinline__ D3 operator*(D3 a, D3 b) {
    return {a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2};
}
__device__ __forceinline__ D3 operator*(double s, D3 a) { return {s * a.v, s * a.d0, s * a.d1, s * a.d2}; }
__device__ __forceinline__ D3 operator+(double s, D3 a) { return {s + a.v, a.d0, a.d1, a.d2}; }
__device__ __forceinline__ D3 operator-(D3 a, double s) { return {a.v - s, a.d0, a.d1, a.d2}; }
__device__ __forceinline__ D3 operator-(double s, D3 a) { return {s - a.v, -a.d0, -a.d1, -a.d2}; }
__device__ __forceinline__ D3 ddiv(D3 a, D3 b) {
    double q = a.v / b.v;
    double ib = 1.0 / b.v;
    return {q, (a.d0 - q * b.d0) * ib, (a.d1 - q * b.d1) * ib, (a.d2 - q * b.d2) * ib};
}
__device__ __forceinline__ D3 dexp(D3 a) {
    double e = exp(a.v);
    return {e, e * a.d0, e * a.d1, e * a.d2};
}
// a^n on a >= 0; an integer exponent 2 avoids pow().
__device__ __forceinline__ D3 dpow(D3 a, double n) {
    double v, dd;
    if (n == 2.0) {
        v = a.v * a.v;
        dd = 2.0 * a.v;
    } else {
        v = pow(a.v, n);
        dd = n * pow(a.v, n - 1.0);
    }
    return {v, dd * a.d0, dd * a.d1, dd * a.d2};
}
// clamp to [0, 1], derivative zero where clamped.
__device__ __forceinline__ D3 dclamp01(D3 a) {
    if (a.v <= 0.0) return dconst(0.0);
    if (a.v >= 1.0) return dconst(1.0);
    return a;
}

}  // namespace bo
