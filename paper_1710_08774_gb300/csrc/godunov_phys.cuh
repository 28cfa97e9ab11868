// godunov_phys.cuh -- per-point device functions of the nine Hydro2D kernels
// (HFAV Sec. 5.4: constoprim, equation_of_state, slope, trace, qleftright,
// riemann, cmpflx, update_cons_vars; make_boundary is the periodic index wrap).
//
// The paper names the kernels only.  The physics is the textbook MUSCL-Hancock
// scheme for the 2D Euler equations of an ideal gas with a two-shock Riemann
// solver (Newton iteration on the star pressure, sampled at x/t = 0).  The
// arithmetic is arranged for a GPU whose FP64 pipe is ~60x slower than FP32:
// every division that can be turned into a product with a reciprocal square
// root is (c = g p s, 1/c = rho s with s = rsqrt(g p rho); 1/W_k and 1/Z_k
// from one rsqrt per side), which changes rounding only.
#pragma once
#include <cuda_runtime.h>

namespace hfav {

#define G_RHO_FLOOR 1e-10
#define G_P_FLOOR 1e-10
#define G_NEWTON_MAX 10
// The iteration stops after an update |dp| <= 1e-8 p*.  Newton converges
// quadratically here, so the error left after that update is of order
// dp^2 / p*, about 1e-16 relative: the same root, to rounding, as a stop at
// 1e-10 (one more iteration on a few faces, which would keep most warps
// iterating for their slowest lane).
#define G_NEWTON_TOL 1e-8
// The FP32-bulk form rounds the star state to FP32 (relative 6e-8), so its
// iteration (still in FP64) stops at |dp| <= 1e-4 p*: the error left, of
// order dp^2 / p*, is about 1e-8, the size of that rounding.  Faces of a
// smooth flow then stop after one update, where the FP64 form takes two.
#define G_NEWTON_TOL_BULK 1e-4

// ---- arithmetic helpers that keep work off the FP64 pipe ------------------
// On this part the FP64 pipe issues ~1/58 of the FP32 rate, so compares,
// floors and sign tests of doubles go through their bit patterns on the
// integer pipe, and reciprocals use the hardware estimate refined by
// Newton-Raphson (each step r <- r + r (1 - b r) squares the relative error;
// the estimate has ~2^-23, two steps reach the last bits of a double).

// x < y for doubles that are not NaN, as signed 64-bit compares of the bits
__device__ __forceinline__ bool dlt(double x, double y) {
    long long a = __double_as_longlong(x), b = __double_as_longlong(y);
    // negative doubles order reversed as integers: flip their magnitude bits
    a ^= (a >> 63) & 0x7fffffffffffffffLL;
    b ^= (b >> 63) & 0x7fffffffffffffffLL;
    return a < b;
}
__device__ __forceinline__ bool dlt(float x, float y) { return x < y; }
// max(x, floor) for a positive floor
__device__ __forceinline__ double dfloor(double x, double fl) { return dlt(x, fl) ? fl : x; }
__device__ __forceinline__ float dfloor(float x, float fl) { return x < fl ? fl : x; }
// |x| < |y|
__device__ __forceinline__ bool dabslt(double x, double y) {
    unsigned long long a = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    unsigned long long b = (unsigned long long)__double_as_longlong(y) & 0x7fffffffffffffffULL;
    return a < b;
}
__device__ __forceinline__ bool dabslt(float x, float y) { return fabsf(x) < fabsf(y); }
// sign classes: > 0, < 0
__device__ __forceinline__ bool dpos(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool dneg(double x) { return __double_as_longlong(x) < 0 && (__double_as_longlong(x) & 0x7fffffffffffffffLL) != 0; }
__device__ __forceinline__ bool dpos(float x) { return x > 0.f; }
// 0 < x < inf (false for NaN): the bit pattern minus one lies below that of the
// largest finite double only for positive finite x
__device__ __forceinline__ bool dposfin(double x) {
    return (unsigned long long)(__double_as_longlong(x) - 1) < 0x7fefffffffffffffULL;
}
__device__ __forceinline__ bool dposfin(float x) { return x > 0.f && x <= 3.402823466e38f; }
__device__ __forceinline__ bool dneg(float x) { return x < 0.f; }

// x / 2, bit for bit the IEEE product x * 0.5, mostly on the integer pipe:
// when x * 0.5 is normal it is x with its exponent field lowered by one (one
// integer subtraction on the high word), zeros pass unchanged, and only the
// rare rest (results that would be subnormal, infinities, NaNs) takes the
// FP64 multiply, out of line.  Every halving of the Godunov arithmetic takes
// this form in FP64, off the FP64 pipe that bounds it.
__device__ __noinline__ double dhalf_rare(double x) { return x * 0.5; }
__device__ __forceinline__ double dhalf(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
    if (e - 2u < 2045u) return __hiloint2double(hi - (1 << 20), lo);   // 2 <= e <= 2046
    if (((hi & 0x7fffffff) | lo) == 0) return x;                         // +-0
    return dhalf_rare(x);
}
__device__ __forceinline__ float dhalf(float x) { return 0.5f * x; }

// FP32 -> FP64 widening on the integer pipe, bit for bit the conversion:
// a normal float keeps its sign, its exponent rebiased (+896) and its
// significand shifted into place; zeros keep their sign; subnormals,
// infinities and NaNs take the conversion instruction, out of line.
__device__ __noinline__ double widen_rare(float x) { return (double)x; }
__device__ __forceinline__ double widen(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    if (e - 1u < 254u)
        return __hiloint2double((int)((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)), (int)(b << 29));
    if ((b & 0x7fffffffu) == 0) return __hiloint2double((int)(b & 0x80000000u), 0);
    return widen_rare(x);
}
__device__ __forceinline__ double widen(double x) { return x; }
// FP64 -> FP32 narrowing on the integer pipe, bit for bit the conversion
// (round to nearest even): a double whose float is normal keeps its sign,
// its exponent rebiased (-896) and its significand's top 23 bits rounded on
// the 29 dropped (a carry into the exponent, up to infinity, is the
// conversion's own); the rest (zeros, float subnormals and underflow,
// infinities, NaNs) takes the conversion instruction, out of line.
__device__ __noinline__ float narrow_rare(double x) { return (float)x; }
__device__ __forceinline__ float narrow(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e - 897u < 254u) {   // 897 <= e <= 1150: float exponent 1 .. 254
        unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu;
        m += (rem > 0x10000000u) | ((rem == 0x10000000u) & (m & 1u));
        return __uint_as_float((hi & 0x80000000u) | (((e - 896u) << 23) + m));
    }
    return narrow_rare(x);
}
// the bulk precision's value of an FP64 intermediate
template <typename T>
__device__ __forceinline__ T to_bulk(double x) {
    if constexpr (sizeof(T) == 4) return narrow(x);
    else return x;
}
// max of a running wave speed and a new one, both non-negative doubles, as
// integers (their order is that of their bits); a NaN speed is passed over,
// as fmax does
__device__ __forceinline__ double speed_max(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    return (ib > ia && ib <= 0x7ff0000000000000LL) ? b : a;
}


// Primitive state of a cell in the frame of a sweep: rho, u_normal,
// u_transverse, p, sound speed c, 1/c and c/rho.
template <typename T>
struct Prim {
    T r, un, ut, p, c, ic, cr;
};

// constoprim + equation_of_state for one cell
template <typename T>
__device__ __forceinline__ Prim<T> cons_to_prim(T U0, T Un, T Ut, T E, T g) {
    Prim<T> w;
    T r = dfloor(U0, (T)G_RHO_FLOOR);
    T ir = rcp_nr(r);
    w.r = r;
    w.un = Un * ir;
    w.ut = Ut * ir;
    T e = fma(E, ir, -dhalf(fma(w.un, w.un, w.ut * w.ut)));
    T p = (g - (T)1) * r * e;
    p = dfloor(p, (T)G_P_FLOOR);
    w.p = p;
    T s = rsqrt(g * p * r);
    w.c = g * p * s;
    w.ic = r * s;
    w.cr = w.c * ir;
    return w;
}

// minmod of two differences: zero unless both have the same strict sign
template <typename T>
__device__ __forceinline__ T minmod(T a, T b) {
    if ((dpos(a) && dpos(b)) || (dneg(a) && dneg(b))) return dabslt(a, b) ? a : b;
    return (T)0;
}

template <typename T>
struct Face4 {
    T r, u, v, p;
};

// trace for one cell: characteristic tracing (MUSCL-Hancock) of the limited
// slopes to the face-left (qm, at a-1/2) and face-right (qp, at a+1/2) states.
template <typename T>
__device__ __forceinline__ void trace(const Prim<T>& w0, T dr, T du, T dv, T dp, T dtdx, Face4<T>& qm,
                                      Face4<T>& qp) {
    const T ic = w0.ic, c = w0.c, r = w0.r, u = w0.un;
    const T dpc = dp * ic;
    const T a1 = dhalf(ic) * fma(-r, du, dpc);
    const T a2 = fma(-dpc, ic, dr);
    const T a3 = dv;
    const T a4 = dhalf(ic) * fma(r, du, dpc);
    const T n1 = (u - c) * dtdx, n2 = u * dtdx, n4 = (u + c) * dtdx;
    // b+ = (1 - nu) a / 2, b- = (1 + nu) a / 2
    const T p1 = dhalf(a1 - n1 * a1), m1 = dhalf(fma(n1, a1, a1));
    const T p2 = dhalf(a2 - n2 * a2), m2 = dhalf(fma(n2, a2, a2));
    const T p3 = dhalf(a3 - n2 * a3), m3 = dhalf(fma(n2, a3, a3));
    const T p4 = dhalf(a4 - n4 * a4), m4 = dhalf(fma(n4, a4, a4));
    const T c2 = c * c;
    qp.r = w0.r + ((p1 + p2) + p4);
    qp.u = fma(w0.cr, p4 - p1, u);
    qp.v = w0.ut + p3;
    qp.p = fma(c2, p1 + p4, w0.p);
    qm.r = w0.r - ((m1 + m2) + m4);
    qm.u = fma(-w0.cr, m4 - m1, u);
    qm.v = w0.ut - m3;
    qm.p = fma(-c2, m1 + m4, w0.p);
}

// slope (minmod-limited differences of the primitives) + trace
template <typename T>
__device__ __forceinline__ void slope_trace(const Prim<T>& wm, const Prim<T>& w0, const Prim<T>& wp, T dtdx,
                                            Face4<T>& qm, Face4<T>& qp) {
    trace(w0, minmod(w0.r - wm.r, wp.r - w0.r), minmod(w0.un - wm.un, wp.un - w0.un),
          minmod(w0.ut - wm.ut, wp.ut - w0.ut), minmod(w0.p - wm.p, wp.p - w0.p), dtdx, qm, qp);
}

// Two-shock Riemann solver: Newton on p* in FP64 (whatever T is), then the
// star state and the sampling at x/t = 0 in T.  Returns the Godunov state.
// FP64 reciprocal square root inside the Newton iteration.  The FP64 form
// calls CUDA's rsqrt.  The FP32-bulk form, whose results are held to the FP32
// bar, takes the hardware estimate (rsqrt.approx.ftz.f64) and one
// Newton-Raphson step y (3 - x y^2) / 2 (a published method): the relative
// error squares to about 2^-38, far below the iteration's 1e-10 tolerance.
template <typename T>
__device__ __forceinline__ double newton_rsqrt(double x) {
    if constexpr (sizeof(T) == 8) {
        return rsqrt(x);
    } else {
        double y;
        asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
        const double e = fma(-x * y, y, 1.0);   // 1 - x y^2
        return fma(dhalf(y), e, y);
    }
}

// ashk = (g + 1) / (2 g), the shock coefficient (computed once on the host);
// nmax: the cap on Newton iterations (G_NEWTON_MAX unless the rule sets one)
template <typename T>
__device__ __forceinline__ Face4<T> riemann(const Face4<T>& L, const Face4<T>& R, T g, double ashk, int nmax,
                                             int* nonconv) {
    const double gd = widen(g);
    const double pl = widen(L.p), pr = widen(R.p), rl = widen(L.r), rr = widen(R.r);
    const double ul = widen(L.u), ur = widen(R.u);
    const double xl = gd * pl * rl, xr = gd * pr * rr;
    const double sl = newton_rsqrt<T>(xl), sr = newton_rsqrt<T>(xr);   // 1 / C_k
    const double cl = xl * sl, cr = xr * sr;               // C_k = sqrt(g p_k rho_k)
    // a / p_k.  The FP32-bulk form takes a g rho_k / C_k^2 from the
    // reciprocal square roots above (2% faster there); the FP64 form keeps
    // one reciprocal of p_L p_R, which does not wait for them (2% faster there)
    double al, ar;
    if constexpr (sizeof(T) == 4) {
        const double ag = ashk * gd;
        al = ag * rl * (sl * sl);
        ar = ag * rr * (sr * sr);
    } else {
        const double ipp = rcp_nr(pl * pr);
        al = ashk * pr * ipp;
        ar = ashk * pl * ipp;
    }
    // initial guess: the acoustic (linearised) star pressure.  The FP32-bulk
    // form takes it in FP32 from its FP32 states: the guess only sets where
    // the FP64 iteration starts, not the root it converges to
    double ps;
    if constexpr (sizeof(T) == 4) {
        const float xlf = g * L.p * L.r, xrf = g * R.p * R.r;
        const float clf = xlf * rsqrtf(xlf), crf = xrf * rsqrtf(xrf);
        ps = widen(fmaxf((crf * L.p + clf * R.p - clf * crf * (R.u - L.u)) / (clf + crf), (float)G_P_FLOOR));
    } else {
        ps = div_nr(cr * pl + cl * pr - cl * cr * (ur - ul), cl + cr);
    }
    ps = dfloor(ps, G_P_FLOOR);
    bool conv = false;
    for (int it = 0; it < nmax; ++it) {
        const double ql = newton_rsqrt<T>(fma(al, ps - pl, 1.0));
        const double qr = newton_rsqrt<T>(fma(ar, ps - pr, 1.0));
        const double iwl = ql * sl, iwr = qr * sr;         // 1 / W_k
        const double izl = dhalf(iwl) * fma(cl * cl, iwl * iwl, 1.0);   // 1 / Z_k
        const double izr = dhalf(iwr) * fma(cr * cr, iwr * iwr, 1.0);
        const double usl = fma(-(ps - pl), iwl, ul);
        const double usr = fma(ps - pr, iwr, ur);
        // the Newton correction itself needs no last-bit accuracy: one
        // refinement of the estimate is enough (the fixed point is set by
        // usr == usl, not by this quotient)
        const double den = izl + izr;
        double rd = rcp_est(den);
        rd = fma(rd, fma(-den, rd, 1.0), rd);
        double pn = fma(-(usr - usl), rd, ps);
        pn = dfloor(pn, G_P_FLOOR);
        conv = !dlt((sizeof(T) == 4 ? G_NEWTON_TOL_BULK : G_NEWTON_TOL) * pn, fabs(pn - ps));
        ps = pn;
        if (conv) break;
    }
    if (!conv) *nonconv = 1;
    // star state at the converged p*, in the bulk precision
    const T pst = to_bulk<T>(ps);
    const T tl = fma(to_bulk<T>(al), pst - L.p, (T)1), tr = fma(to_bulk<T>(ar), pst - R.p, (T)1);
    const T qlt = rsqrt(tl), qrt = rsqrt(tr);
    const T Cl = to_bulk<T>(cl), Cr = to_bulk<T>(cr);
    const T wl = Cl * tl * qlt, wr = Cr * tr * qrt;        // W_k = C_k sqrt(t_k)
    const T iwl = qlt * to_bulk<T>(sl), iwr = qrt * to_bulk<T>(sr);
    const T ust = div_nr(fma(wl, L.u, wr * R.u) + (L.p - R.p), wl + wr);
    const bool left = dpos(ust);
    const Face4<T>& S = left ? L : R;
    const T ws = left ? wl : wr, iws = left ? iwl : iwr;
    const T sgn = left ? (T)-1 : (T)1;
    T rst = div_nr(S.r, fma(-S.r * (pst - S.p), iws * iws, (T)1));
    rst = dfloor(rst, (T)G_RHO_FLOOR);
    Face4<T> o;
    o.v = S.v;
    bool take_side, take_star;
    T f = (T)0;
    if (dlt(S.p, pst)) {   // shock: it has passed the face when sgn * S < 0
        take_side = dneg(fma(sgn * S.u, S.r, ws));
        take_star = !take_side;
    } else {           // rarefaction fan
        // The head u_s + sgn c_s has passed the face when the side's flow
        // is supersonic away from the contact (sgn u_s < 0 and u_s^2 > c_s^2),
        // and the tail u* + sgn c* has not reached it when the star flow is
        // subsonic (u*^2 < c*^2; sgn u* <= 0 on the sampled side): squared
        // speeds, so no sound speed is needed unless the face lies inside the
        // fan.  At the fan's edges the state is continuous, so a decision
        // that rounding flips there moves it by rounding only.
        const T gps = g * S.p, gpst = g * pst;
        take_side = (left ? dpos(S.u) : dneg(S.u)) && dlt(gps, S.r * S.u * S.u);
        take_star = !take_side && dlt(rst * ust * ust, gpst);
        if (!take_side && !take_star) {   // inside the fan: interpolate between its edges
            const T cs = gps * rsqrt(gps * S.r);
            const T cst = gpst * rsqrt(gpst * rst);
            const T head = fma(sgn, cs, S.u);
            const T tail = fma(sgn, cst, ust);
            if (head == tail) take_star = true;   // degenerate fan
            else f = div_nr(-tail, head - tail);
        }
    }
    if (take_side) { o.r = S.r; o.u = S.u; o.p = S.p; }
    else if (take_star) { o.r = rst; o.u = ust; o.p = pst; }
    else {
        o.r = fma(f, S.r - rst, rst);
        o.u = fma(f, S.u - ust, ust);
        o.p = fma(f, S.p - pst, pst);
    }
    return o;
}

// cmpflx: Euler flux through the face of the Godunov state
template <typename T>
__device__ __forceinline__ Face4<T> flux(const Face4<T>& q, T ig1) {
    Face4<T> F;
    const T m = q.r * q.u;
    F.r = m;
    F.u = fma(m, q.u, q.p);
    F.v = m * q.v;
    const T et = fma(q.p, ig1, dhalf(q.r) * fma(q.u, q.u, q.v * q.v));
    F.p = q.u * (et + q.p);
    return F;
}

// CFL wave speed max(|u|+c, |v|+c) of a conserved state, in FP64; also flags
// non-physical states (rho <= 0 or p <= 0 before any floor)
__device__ __forceinline__ double wave_speed(double U0, double U1, double U2, double U3, double g, int* bad) {
    const double ir = rcp_nr(U0);
    const double u = U1 * ir, v = U2 * ir;
    const double e = fma(U3, ir, -dhalf(fma(u, u, v * v)));
    double p = (g - 1.0) * U0 * e;
    if (!dposfin(U0) || !dposfin(p)) *bad = 1;   // also NaN and infinite states
    p = dfloor(p, G_P_FLOOR);
    const double c = g * p * rsqrt(g * p * U0);
    return (dabslt(u, v) ? fabs(v) : fabs(u)) + c;
}

// Same in FP32 for the FP32 bulk mode (the reduction itself is FP64)
__device__ __forceinline__ double wave_speed(float U0, float U1, float U2, float U3, float g, int* bad) {
    const float ir = 1.0f / U0;
    const float u = U1 * ir, v = U2 * ir;
    const float e = fmaf(U3, ir, -0.5f * fmaf(u, u, v * v));
    float p = (g - 1.0f) * U0 * e;
    if (!dposfin(U0) || !dposfin(p)) *bad = 1;
    p = fmaxf(p, (float)G_P_FLOOR);
    const float c = g * p * rsqrtf(g * p * U0);
    return widen(fmaxf(fabsf(u), fabsf(v)) + c);
}

}  // namespace hfav
