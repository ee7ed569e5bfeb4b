// Host-side dual numbers (Sec. 2, Eqs. 1-4) and the dual transfer maps of
// Sec. 4 (Eq. "quadtr" and its defocusing twin) used to build the per-kick
// coefficient tables of the PIC runtimes. FP64, 16 channels (value and up to
// 15 derivatives); unused channels stay zero.
#pragma once
#include <cmath>

namespace adpic_host {

constexpr int kMaxCP = 16;

// ------------------------------------------------------------------ host dual numbers
// value v[0] and derivatives v[1..]; all 16 slots are carried, unused ones stay 0
struct HD {
    double v[kMaxCP];
};
inline HD hc(double x) { HD r{}; r.v[0] = x; return r; }
inline HD hvar(double x, int slot) { HD r = hc(x); if (slot >= 0) r.v[slot + 1] = 1.0; return r; }
inline HD hadd(const HD& a, const HD& b) { HD r; for (int k = 0; k < kMaxCP; ++k) r.v[k] = a.v[k] + b.v[k]; return r; }
inline HD hneg(const HD& a) { HD r; for (int k = 0; k < kMaxCP; ++k) r.v[k] = -a.v[k]; return r; }
inline HD hmul(const HD& a, const HD& b) {           // Eq. 2
    HD r;
    r.v[0] = a.v[0] * b.v[0];
    for (int k = 1; k < kMaxCP; ++k) r.v[k] = b.v[0] * a.v[k] + a.v[0] * b.v[k];
    return r;
}
inline HD hdiv(const HD& a, const HD& b) {           // Eq. 3
    HD r;
    r.v[0] = a.v[0] / b.v[0];
    for (int k = 1; k < kMaxCP; ++k) r.v[k] = (a.v[k] * b.v[0] - b.v[k] * a.v[0]) / (b.v[0] * b.v[0]);
    return r;
}
inline HD hfn(const HD& a, double h, double hp) {    // Eq. 4
    HD r;
    r.v[0] = h;
    for (int k = 1; k < kMaxCP; ++k) r.v[k] = hp * a.v[k];
    return r;
}
inline HD hsqrt(const HD& a) { double s = std::sqrt(a.v[0]); return hfn(a, s, 0.5 / s); }
inline HD hsin(const HD& a) { return hfn(a, std::sin(a.v[0]), std::cos(a.v[0])); }
inline HD hcos(const HD& a) { return hfn(a, std::cos(a.v[0]), -std::sin(a.v[0])); }
inline HD hsinh(const HD& a) { return hfn(a, std::sinh(a.v[0]), std::cosh(a.v[0])); }
inline HD hcosh(const HD& a) { return hfn(a, std::cosh(a.v[0]), std::sinh(a.v[0])); }

struct HMap { HD m[3][4]; };   // per plane (m11, m12, m21, m22)

// one transverse plane over step t with focusing strength kp (Sec. 4: cos/sin
// in the focusing plane, cosh/sinh in the defocusing plane, drift at kp = 0)
inline void plane_map(const HD& kp, const HD& t, HD* m) {
    if (kp.v[0] > 0.0) {
        HD w = hsqrt(kp), th = hmul(w, t), c = hcos(th), s = hsin(th);
        m[0] = c; m[1] = hdiv(s, w); m[2] = hneg(hmul(w, s)); m[3] = c;
    } else if (kp.v[0] < 0.0) {
        HD w = hsqrt(hneg(kp)), th = hmul(w, t), c = hcosh(th), s = hsinh(th);
        m[0] = c; m[1] = hdiv(s, w); m[2] = hmul(w, s); m[3] = c;
    } else {
        m[0] = hc(1.0); m[1] = t; m[2] = hc(0.0); m[3] = hc(1.0);
    }
}

inline HMap compose(const HMap& B, const HMap& A) {   // B after A
    HMap r;
    for (int p = 0; p < 3; ++p) {
        const HD* a = A.m[p];
        const HD* b = B.m[p];
        r.m[p][0] = hadd(hmul(b[0], a[0]), hmul(b[1], a[2]));
        r.m[p][1] = hadd(hmul(b[0], a[1]), hmul(b[1], a[3]));
        r.m[p][2] = hadd(hmul(b[2], a[0]), hmul(b[3], a[2]));
        r.m[p][3] = hadd(hmul(b[2], a[1]), hmul(b[3], a[3]));
    }
    return r;
}


}  // namespace adpic_host
