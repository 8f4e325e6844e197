// Device-side helpers shared by the CUDA translation units of libhm:
// complex FP64 arithmetic, the cube-mapped ellipsoid patch map and its inverse
// chart, Chebyshev polynomials.  (Sec. II.B, Eqs. 11-14.)
#pragma once
#include <cuda_runtime.h>
#include <math.h>

typedef double2 zc;  // complex128: x = re, y = im
typedef float2 cf;   // complex64

// Real type of a complex storage type.
template <class C> struct CReal;
template <> struct CReal<double2> { typedef double R; };
template <> struct CReal<float2> { typedef float R; };

// Complex arithmetic, generic over complex64 / complex128 storage.
__host__ __device__ __forceinline__ zc zmake(double r, double i) { return make_double2(r, i); }
template <class C>
__host__ __device__ __forceinline__ C cmk(typename CReal<C>::R r, typename CReal<C>::R i)
{
    C c;
    c.x = r;
    c.y = i;
    return c;
}
template <class C> __host__ __device__ __forceinline__ C zadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <class C> __host__ __device__ __forceinline__ C zsub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <class C> __host__ __device__ __forceinline__ C zmul(C a, C b)
{
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class C> __host__ __device__ __forceinline__ C zconj(C a) { return cmk<C>(a.x, -a.y); }
template <class C> __host__ __device__ __forceinline__ C zscale(C a, typename CReal<C>::R s)
{
    return cmk<C>(a.x * s, a.y * s);
}
template <class C> __host__ __device__ __forceinline__ typename CReal<C>::R zabs2(C a) { return a.x * a.x + a.y * a.y; }
// a += b * c
template <class C> __host__ __device__ __forceinline__ C zfma(C b, C c, C a)
{
    return cmk<C>(fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y)));
}
// a += conj(b) * c
template <class C> __host__ __device__ __forceinline__ C zfmac(C b, C c, C a)
{
    return cmk<C>(fma(b.x, c.x, fma(b.y, c.y, a.x)), fma(b.x, c.y, fma(-b.y, c.x, a.y)));
}
template <class C> __device__ __forceinline__ C zdiv(C a, C b)
{
    typename CReal<C>::R s = (typename CReal<C>::R)1 / (b.x * b.x + b.y * b.y);
    return cmk<C>((a.x * b.x + a.y * b.y) * s, (a.y * b.x - a.x * b.y) * s);
}
// Conversions between the two storage precisions.
__host__ __device__ __forceinline__ void cconv(double2 a, double2 &o) { o = a; }
__host__ __device__ __forceinline__ void cconv(double2 a, float2 &o) { o = make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ void cconv(float2 a, double2 &o) { o = make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ void cconv(float2 a, float2 &o) { o = a; }

// One body (cube-mapped ellipsoid): r = c + M xhat, M = Rot diag(semi), Minv = M^-1.
struct DevBody {
    double c[3];
    double M[9];
    double Minv[9];
    int m;
    int pad;
};
// One patch: body, cube face, sub-square (i, j).
struct DevPatch {
    int body, face, i, j;
};

// Face frames (e_f, e1, e2), e1 x e2 = e_f so a_u x a_v is the outward normal.
__host__ __device__ __forceinline__ void face_frame(int f, double *ef, double *e1, double *e2)
{
    ef[0] = ef[1] = ef[2] = 0.0;
    e1[0] = e1[1] = e1[2] = 0.0;
    e2[0] = e2[1] = e2[2] = 0.0;
    switch (f) {
    case 0: ef[0] = 1; e1[1] = 1; e2[2] = 1; break;
    case 1: ef[0] = -1; e1[2] = 1; e2[1] = 1; break;
    case 2: ef[1] = 1; e1[2] = 1; e2[0] = 1; break;
    case 3: ef[1] = -1; e1[0] = 1; e2[2] = 1; break;
    case 4: ef[2] = 1; e1[0] = 1; e2[1] = 1; break;
    default: ef[2] = -1; e1[1] = 1; e2[0] = 1; break;
    }
}

// r(u,v), a_u = dr/du, a_v = dr/dv for patch P of body B (Eq. 14); equiangular cube map.
__host__ __device__ __forceinline__ void patch_eval(const DevBody &B, const DevPatch &P, double u, double v,
                                           double *r, double *ru, double *rv)
{
    const double q = 0.78539816339744830962;  // pi/4
    double ef[3], e1[3], e2[3];
    face_frame(P.face, ef, e1, e2);
    double im = 1.0 / B.m;
    double s = -1.0 + (2.0 * P.i + 1.0 + u) * im;
    double t = -1.0 + (2.0 * P.j + 1.0 + v) * im;
    double S = tan(q * s), T = tan(q * t);
    double dS = q * (1.0 + S * S) * im, dT = q * (1.0 + T * T) * im;
    double c0 = ef[0] + S * e1[0] + T * e2[0];
    double c1 = ef[1] + S * e1[1] + T * e2[1];
    double c2 = ef[2] + S * e1[2] + T * e2[2];
    double n2 = c0 * c0 + c1 * c1 + c2 * c2;
    double in = 1.0 / sqrt(n2);
    double in3 = in * in * in;
    double cu0 = dS * e1[0], cu1 = dS * e1[1], cu2 = dS * e1[2];
    double cv0 = dT * e2[0], cv1 = dT * e2[1], cv2 = dT * e2[2];
    double ccu = c0 * cu0 + c1 * cu1 + c2 * cu2, ccv = c0 * cv0 + c1 * cv1 + c2 * cv2;
    double xh[3] = {c0 * in, c1 * in, c2 * in};
    double xu[3] = {cu0 * in - c0 * ccu * in3, cu1 * in - c1 * ccu * in3, cu2 * in - c2 * ccu * in3};
    double xv[3] = {cv0 * in - c0 * ccv * in3, cv1 * in - c1 * ccv * in3, cv2 * in - c2 * ccv * in3};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double *Ma = B.M + 3 * a;
        r[a] = B.c[a] + Ma[0] * xh[0] + Ma[1] * xh[1] + Ma[2] * xh[2];
        ru[a] = Ma[0] * xu[0] + Ma[1] * xu[1] + Ma[2] * xu[2];
        rv[a] = Ma[0] * xv[0] + Ma[1] * xv[1] + Ma[2] * xv[2];
    }
}

// Chart coordinates (u, v) of a surface point x in patch P's extended chart.
// Returns false when x is not in the half-space of P's cube face (chart undefined).
__host__ __device__ __forceinline__ bool patch_chart(const DevBody &B, const DevPatch &P, const double *x,
                                            double *u, double *v)
{
    double d[3] = {x[0] - B.c[0], x[1] - B.c[1], x[2] - B.c[2]};
    double y[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) y[a] = B.Minv[3 * a] * d[0] + B.Minv[3 * a + 1] * d[1] + B.Minv[3 * a + 2] * d[2];
    double ef[3], e1[3], e2[3];
    face_frame(P.face, ef, e1, e2);
    double yn = y[0] * ef[0] + y[1] * ef[1] + y[2] * ef[2];
    if (!(yn > 1e-12)) return false;
    double S = (y[0] * e1[0] + y[1] * e1[1] + y[2] * e1[2]) / yn;
    double T = (y[0] * e2[0] + y[1] * e2[1] + y[2] * e2[2]) / yn;
    const double iq = 1.27323954473516268615;  // 4/pi
    double s = iq * atan(S), t = iq * atan(T);
    *u = B.m * (s + 1.0) - (2.0 * P.i + 1.0);
    *v = B.m * (t + 1.0) - (2.0 * P.j + 1.0);
    return true;
}

// T_0..T_{n-1} at x by the three-term recurrence.
__host__ __device__ __forceinline__ void cheb_T(int n, double x, double *t)
{
    t[0] = 1.0;
    if (n > 1) t[1] = x;
    for (int j = 2; j < n; ++j) t[j] = 2.0 * x * t[j - 1] - t[j - 2];
}

#define HM_NC_MAX 16
