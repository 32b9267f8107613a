// Site arithmetic of the H_w(mu) stencil (Eq. 2), generic in the number type.
//
// (D_w psi)_n = psi_n - kappa sum_nu [ w+_nu (1+gamma_nu) U_{n,nu} psi_{n+nu}
//                                     + w-_nu (1-gamma_nu) U^dag_{n-nu,nu} psi_{n-nu} ]
// with w+-_4 = e^{+-mu} on the time hops and 1 otherwise. In the chiral basis
// (gamma_5 = diag(1,1,-1,-1)) each projector (1 +- gamma_nu) has rank 2: the
// hop projects the neighbour to a half spinor (2 spins x 3 colours),
// multiplies it by the link (two SU(3) mat-vecs instead of four) and expands
// it back; spins 2,3 of the expansion are fixed multiples of spins 0,1.
//
// Every function here is __host__ __device__: the kernels of dslash.cu run
// them on the GPU, and a host build runs the same arithmetic on the CPU so
// that it can be checked there (loads go through OVL_LDG: __ldg on the device,
// a plain load on the host). T is the arithmetic type (double, float, or the
// double-float dd of dd.cuh), VT the stored spinor element (double2 / float2).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>

#include <cmath>

#include "../../include/ovl.h"

#define OVL_HD __host__ __device__ __forceinline__
#ifdef __CUDA_ARCH__
#define OVL_LDG(p) __ldg(p)
#else
#define OVL_LDG(p) (*(p))
#endif

namespace ovl_stencil {

// fused multiply-add of the plain types (the dd overload is in dd.cuh)
OVL_HD double ffma(double a, double b, double c) {
#ifdef __CUDA_ARCH__
    return fma(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}
OVL_HD float ffma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return fmaf(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}

template <typename T>
struct C {
    T r, i;
};
template <typename T>
OVL_HD C<T> mk(T r, T i) {
    return C<T>{r, i};
}
template <typename T>
OVL_HD C<T> operator+(C<T> a, C<T> b) {
    return {a.r + b.r, a.i + b.i};
}
template <typename T>
OVL_HD C<T> operator-(C<T> a, C<T> b) {
    return {a.r - b.r, a.i - b.i};
}
template <typename T>
OVL_HD C<T> operator*(C<T> a, C<T> b) {
    return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename T>
OVL_HD C<T> operator*(T s, C<T> a) {
    return {s * a.r, s * a.i};
}
template <typename T>
OVL_HD C<T> conj(C<T> a) {
    return {a.r, -a.i};
}
template <typename T>
OVL_HD C<T> ti(C<T> a) {  // i * a
    return {-a.i, a.r};
}
template <typename T>
OVL_HD C<T> tmi(C<T> a) {  // -i * a
    return {a.i, -a.r};
}
// a * b + c
template <typename T>
OVL_HD C<T> cfma(C<T> a, C<T> b, C<T> c) {
    c.r = ffma(a.r, b.r, c.r);
    c.r = ffma(-a.i, b.i, c.r);
    c.i = ffma(a.r, b.i, c.i);
    c.i = ffma(a.i, b.r, c.i);
    return c;
}
// conj(a) * b + c
template <typename T>
OVL_HD C<T> cjfma(C<T> a, C<T> b, C<T> c) {
    c.r = ffma(a.r, b.r, c.r);
    c.r = ffma(a.i, b.i, c.r);
    c.i = ffma(a.r, b.i, c.i);
    c.i = ffma(-a.i, b.r, c.i);
    return c;
}

struct KArgs {
    const void* const* in;
    void* const* out;
    const double* mu;
    const int* active;
    const int* klim;
    int stride, j;
    int Lx, Ly, Lz, Lt;
    // site tiling of a CTA: tx x ty x tz sites (x fastest) at one t, so that
    // the neighbour spinors a CTA reads are mostly loaded by the CTA itself
    // (L1 hits); tx == 0: consecutive site indices per CTA
    int tx, ty, tz;
    size_t V;
    double kappa;
    int apbc;
    const double2* u64;
    const float4* u32q;
    const float2* u32r;
    const float4* u12;
};

// load the 12 components of a packed spinor at a site
template <typename T, typename VT>
OVL_HD void load_spinor(const VT* __restrict__ p, size_t V, size_t s, C<T> (&psi)[12]) {
#pragma unroll
    for (int cp = 0; cp < 6; cp++) {
        if constexpr (sizeof(VT) == sizeof(double2)) {
            const double2* q = (const double2*)p + ((size_t)cp * V + s) * 2;
            double2 a = OVL_LDG(q), b = OVL_LDG(q + 1);
            psi[2 * cp] = mk<T>((T)a.x, (T)a.y);
            psi[2 * cp + 1] = mk<T>((T)b.x, (T)b.y);
        } else {
            float4 a = OVL_LDG((const float4*)p + ((size_t)cp * V + s));
            psi[2 * cp] = mk<T>((T)a.x, (T)a.y);
            psi[2 * cp + 1] = mk<T>((T)a.z, (T)a.w);
        }
    }
}

template <typename T, typename VT>
OVL_HD void store_spinor(VT* __restrict__ p, size_t V, size_t s, const C<T> (&o)[12]) {
#pragma unroll
    for (int cp = 0; cp < 6; cp++) {
        if constexpr (sizeof(VT) == sizeof(double2)) {
            double2* q = (double2*)p + ((size_t)cp * V + s) * 2;
            q[0] = make_double2((double)o[2 * cp].r, (double)o[2 * cp].i);
            q[1] = make_double2((double)o[2 * cp + 1].r, (double)o[2 * cp + 1].i);
        } else {
            ((float4*)p)[(size_t)cp * V + s] =
                make_float4((float)o[2 * cp].r, (float)o[2 * cp].i, (float)o[2 * cp + 1].r, (float)o[2 * cp + 1].i);
        }
    }
}

template <typename T, int LINKS>
OVL_HD void load_link(const KArgs& a, int nu, size_t s, C<T> (&u)[9]) {
    const size_t V = a.V;
    if constexpr (LINKS == OVL_LINKS_F64) {
#pragma unroll
        for (int e = 0; e < 9; e++) {
            double2 v = OVL_LDG(a.u64 + ((size_t)nu * 9 + e) * V + s);
            u[e] = mk<T>((T)v.x, (T)v.y);
        }
    } else if constexpr (LINKS == OVL_LINKS_F32) {
#pragma unroll
        for (int p = 0; p < 4; p++) {
            float4 v = OVL_LDG(a.u32q + ((size_t)nu * 4 + p) * V + s);
            u[2 * p] = mk<T>((T)v.x, (T)v.y);
            u[2 * p + 1] = mk<T>((T)v.z, (T)v.w);
        }
        float2 v = OVL_LDG(a.u32r + (size_t)nu * V + s);
        u[8] = mk<T>((T)v.x, (T)v.y);
    } else {
#pragma unroll
        for (int p = 0; p < 3; p++) {
            float4 v = OVL_LDG(a.u12 + ((size_t)nu * 3 + p) * V + s);
            u[2 * p] = mk<T>((T)v.x, (T)v.y);
            u[2 * p + 1] = mk<T>((T)v.z, (T)v.w);
        }
        // SU(3): third row = complex conjugate of (row 0) x (row 1)
        u[6] = conj(u[1] * u[5] - u[2] * u[4]);
        u[7] = conj(u[2] * u[3] - u[0] * u[5]);
        u[8] = conj(u[0] * u[4] - u[1] * u[3]);
    }
}

// Spin projection (1 + sgn*gamma_nu) psi -> half spinor h0, h1 (colour vectors),
// and the expansion of the two multiplied half spinors back to four spins.
// Component index of psi: 3*spin + colour.
template <typename T, int NU, bool FWD>
OVL_HD void project(const C<T> (&psi)[12], C<T> (&h)[6]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        C<T> p0 = psi[c], p1 = psi[3 + c], p2 = psi[6 + c], p3 = psi[9 + c];
        if constexpr (NU == 0) {  // gamma_x: (g psi) = (i p3, i p2, -i p1, -i p0)
            h[c] = FWD ? p0 + ti(p3) : p0 - ti(p3);
            h[3 + c] = FWD ? p1 + ti(p2) : p1 - ti(p2);
        } else if constexpr (NU == 1) {  // gamma_y: (-p3, p2, p1, -p0)
            h[c] = FWD ? p0 - p3 : p0 + p3;
            h[3 + c] = FWD ? p1 + p2 : p1 - p2;
        } else if constexpr (NU == 2) {  // gamma_z: (i p2, -i p3, -i p0, i p1)
            h[c] = FWD ? p0 + ti(p2) : p0 - ti(p2);
            h[3 + c] = FWD ? p1 - ti(p3) : p1 + ti(p3);
        } else {  // gamma_t: (p2, p3, p0, p1)
            h[c] = FWD ? p0 + p2 : p0 - p2;
            h[3 + c] = FWD ? p1 + p3 : p1 - p3;
        }
    }
}

// w multiplies the time hops only (NU == 3); a spatial hop's weight is 1
template <typename T, int NU, bool FWD>
OVL_HD void expand_add(const C<T> (&g)[6], T w, C<T> (&acc)[12]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        C<T> g0 = g[c], g1 = g[3 + c];
        if constexpr (NU == 3) {
            g0 = w * g0;
            g1 = w * g1;
        }
        acc[c] = acc[c] + g0;
        acc[3 + c] = acc[3 + c] + g1;
        C<T> r2, r3;
        if constexpr (NU == 0) {
            r2 = FWD ? tmi(g1) : ti(g1);
            r3 = FWD ? tmi(g0) : ti(g0);
        } else if constexpr (NU == 1) {
            r2 = FWD ? g1 : mk<T>(-g1.r, -g1.i);
            r3 = FWD ? mk<T>(-g0.r, -g0.i) : g0;
        } else if constexpr (NU == 2) {
            r2 = FWD ? tmi(g0) : ti(g0);
            r3 = FWD ? ti(g1) : tmi(g1);
        } else {
            r2 = FWD ? g0 : mk<T>(-g0.r, -g0.i);
            r3 = FWD ? g1 : mk<T>(-g1.r, -g1.i);
        }
        acc[6 + c] = acc[6 + c] + r2;
        acc[9 + c] = acc[9 + c] + r3;
    }
}

// g = U h (forward hop) or U^dag h (backward hop) for both spins of the half
// spinor; dd.cuh specialises it for the double-float type
template <typename T>
struct LinkMul {
    template <bool FWD>
    static OVL_HD void run(const C<T> (&u)[9], const C<T> (&h)[6], C<T> (&g)[6]) {
#pragma unroll
        for (int s = 0; s < 2; s++) {
#pragma unroll
            for (int ai = 0; ai < 3; ai++) {
                C<T> z = mk<T>(0, 0);
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    if constexpr (FWD)
                        z = cfma(u[3 * ai + b], h[3 * s + b], z);  // U h
                    else
                        z = cjfma(u[3 * b + ai], h[3 * s + b], z);  // U^dag h
                }
                g[3 * s + ai] = z;
            }
        }
    }
};

template <typename T, typename VT, int LINKS, int NU, bool FWD>
OVL_HD void hop(const KArgs& a, const VT* __restrict__ in, size_t site, size_t nb, T w, C<T> (&acc)[12]) {
    C<T> psi[12];
    load_spinor<T, VT>(in, a.V, nb, psi);
    C<T> h[6];
    project<T, NU, FWD>(psi, h);
    C<T> u[9];
    load_link<T, LINKS>(a, NU, FWD ? site : nb, u);
    C<T> g[6];
    LinkMul<T>::template run<FWD>(u, h, g);
    expand_add<T, NU, FWD>(g, w, acc);
}

// (H_w psi) at one site: the eight hops, psi - kappa * sum, then gamma_5.
// wp, wm: e^{+mu}, e^{-mu} of this right-hand side (the antiperiodic sign of
// the time boundary is applied here).
template <typename T, typename VT, int LINKS>
OVL_HD void site_compute(const KArgs& a, const VT* __restrict__ in, VT* __restrict__ out, size_t site, T wp,
                         T wm) {
    const int Lx = a.Lx, Ly = a.Ly, Lz = a.Lz, Lt = a.Lt;
    const size_t sy = Lx, sz = (size_t)Lx * Ly, st = sz * Lz;
    unsigned q = (unsigned)site;  // V < 2^31 (checked when the lattice is created)
    const int x = (int)(q % (unsigned)Lx);
    q /= (unsigned)Lx;
    const int y = (int)(q % (unsigned)Ly);
    q /= (unsigned)Ly;
    const int z = (int)(q % (unsigned)Lz);
    const int t = (int)(q / (unsigned)Lz);
    const size_t xp = x + 1 == Lx ? site - (Lx - 1) : site + 1;
    const size_t xm = x == 0 ? site + (Lx - 1) : site - 1;
    const size_t yp = y + 1 == Ly ? site - (Ly - 1) * sy : site + sy;
    const size_t ym = y == 0 ? site + (Ly - 1) * sy : site - sy;
    const size_t zp = z + 1 == Lz ? site - (Lz - 1) * sz : site + sz;
    const size_t zm = z == 0 ? site + (Lz - 1) * sz : site - sz;
    const size_t tp = t + 1 == Lt ? site - (Lt - 1) * st : site + st;
    const size_t tm = t == 0 ? site + (Lt - 1) * st : site - st;
    T wtp = wp, wtm = wm;
    if (a.apbc) {
        if (t + 1 == Lt) wtp = -wtp;
        if (t == 0) wtm = -wtm;
    }
    C<T> acc[12];
#pragma unroll
    for (int i = 0; i < 12; i++) acc[i] = mk<T>(0, 0);
    hop<T, VT, LINKS, 0, true>(a, in, site, xp, (T)1, acc);
    hop<T, VT, LINKS, 0, false>(a, in, site, xm, (T)1, acc);
    hop<T, VT, LINKS, 1, true>(a, in, site, yp, (T)1, acc);
    hop<T, VT, LINKS, 1, false>(a, in, site, ym, (T)1, acc);
    hop<T, VT, LINKS, 2, true>(a, in, site, zp, (T)1, acc);
    hop<T, VT, LINKS, 2, false>(a, in, site, zm, (T)1, acc);
    hop<T, VT, LINKS, 3, true>(a, in, site, tp, wtp, acc);
    hop<T, VT, LINKS, 3, false>(a, in, site, tm, wtm, acc);
    C<T> psi[12];
    load_spinor<T, VT>(in, a.V, site, psi);
    const T kap = (T)a.kappa;
    C<T> o[12];
#pragma unroll
    for (int i = 0; i < 12; i++) {
        C<T> d = psi[i] - kap * acc[i];
        o[i] = i < 6 ? d : mk<T>(-d.r, -d.i);  // gamma_5 = diag(1,1,-1,-1)
    }
    store_spinor<T, VT>(out, a.V, site, o);
}

}  // namespace ovl_stencil
