// vspec_radix.cuh — complex helpers and small in-register DFTs.
//
// An element is either one complex value (float2: re, im) or the two
// polarisations of the same sample or channel (float4: x.re, x.im, y.re,
// y.im). Every butterfly applies the same arithmetic to both halves of a
// float4, so both polarisations share twiddle loads and index arithmetic.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

namespace vspec {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float4 cadd(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 csub(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

// (a.re + i a.im) * (w.re + i w.im)
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ float4 cmul(float4 a, float2 w) {
    return make_float4(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x),
                       fmaf(a.z, w.x, -a.w * w.y), fmaf(a.z, w.y, a.w * w.x));
}

// multiplication by -i: (re, im) -> (im, -re)
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }
__device__ __forceinline__ float4 cmul_mi(float4 a) { return make_float4(a.y, -a.x, a.w, -a.z); }

// a + (-i) b and a - (-i) b
template <typename T> __device__ __forceinline__ T add_mi(T a, T b) { return cadd(a, cmul_mi(b)); }
template <typename T> __device__ __forceinline__ T sub_mi(T a, T b) { return csub(a, cmul_mi(b)); }

// Both polarisations of one complex value, packed for the paired FP32
// instructions of sm_100 and later (FADD2 / FMUL2 / FFMA2): re = (X.re, Y.re),
// im = (X.im, Y.im). Every DFT step applies the same operation with the same
// twiddle to X and Y, so each step is one paired instruction for both. In
// memory a P2 is 16 bytes: X.re, Y.re, X.im, Y.im.
struct __align__(16) P2 {
    float2 re, im;
};
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one fused multiply-add with -1 (exactly the rounded difference)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ P2 make_p2(float xr, float xi, float yr, float yi) {
    return P2{make_float2(xr, yr), make_float2(xi, yi)};
}
__device__ __forceinline__ P2 cadd(P2 a, P2 b) { return P2{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ P2 csub(P2 a, P2 b) { return P2{sub2(a.re, b.re), sub2(a.im, b.im)}; }
// (re + i im) (w.x + i w.y) for both polarisations. Scalar multiply-adds: a
// twiddle loaded at run time would first have to be copied into register
// pairs for the paired instructions, which costs more than it saves
// (measured: row and column kernels 1.5-4% faster this way).
__device__ __forceinline__ P2 cmul(P2 a, float2 w) {
    return P2{make_float2(fmaf(a.re.x, w.x, -a.im.x * w.y), fmaf(a.re.y, w.x, -a.im.y * w.y)),
              make_float2(fmaf(a.re.x, w.y, a.im.x * w.x), fmaf(a.re.y, w.y, a.im.y * w.x))};
}
template <> __device__ __forceinline__ P2 add_mi<P2>(P2 a, P2 b) { return P2{add2(a.re, b.im), sub2(a.im, b.re)}; }
template <> __device__ __forceinline__ P2 sub_mi<P2>(P2 a, P2 b) { return P2{sub2(a.re, b.im), add2(a.im, b.re)}; }

// multiplication by a twiddle given as compile-time constants (c, s): c + i s
template <typename T> __device__ __forceinline__ T cmulc(T a, float c, float s) {
    return cmul(a, make_float2(c, s));
}

// Constants: cos and sin of multiples of pi/8 (the 16th roots of unity).
constexpr float kC8 = 0.70710678118654752440f;  // cos(pi/4)
constexpr float kC16 = 0.92387953251128675613f; // cos(pi/8)
constexpr float kS16 = 0.38268343236508977173f; // sin(pi/8)

// A rotation by a compile-time constant c + i s on both polarisations at once:
// (re + i im)(c + i s) = (re c - im s) + i (re s + im c) as four paired
// instructions (the scalar form takes eight); the constant pairs are
// immediates the compiler materialises.
template <int QQ> __device__ __forceinline__ P2 rot_p2(P2 a) {
    constexpr float c16[8] = {1.f, kC16, kC8, kS16, 0.f, -kS16, -kC8, -kC16};   // cos(q pi / 8)
    constexpr float s16[8] = {0.f, -kS16, -kC8, -kC16, -1.f, -kC16, -kC8, -kS16};  // -sin(q pi / 8)
    constexpr float c = c16[QQ], s = s16[QQ];
    if constexpr (QQ == 2 || QQ == 6) {
        // c = +-s: (re + i im)(c + i s) with |c| = |s| = 1/sqrt 2
        if constexpr (QQ == 2) {  // c = kC8, s = -kC8: kC8 ((re + im) + i (im - re))
            const float2 k = make_float2(kC8, kC8);
            return P2{__fmul2_rn(__fadd2_rn(a.re, a.im), k), __fmul2_rn(sub2(a.im, a.re), k)};
        } else {                  // c = s = -kC8: kC8 ((im - re) - i (re + im))
            const float2 k = make_float2(kC8, kC8), nk = make_float2(-kC8, -kC8);
            return P2{__fmul2_rn(sub2(a.im, a.re), k), __fmul2_rn(__fadd2_rn(a.re, a.im), nk)};
        }
    } else {
        const float2 cc = make_float2(c, c), ss = make_float2(s, s), ns = make_float2(-s, -s);
        return P2{__ffma2_rn(a.re, cc, __fmul2_rn(a.im, ns)), __ffma2_rn(a.im, cc, __fmul2_rn(a.re, ss))};
    }
}

// W_R^q = exp(-2 pi i q / R) applied to a, for R in {8, 16}.
template <int R, int Q, typename T> __device__ __forceinline__ T twiddle_const(T a) {
    static_assert(R == 8 || R == 16, "constant twiddles for R = 8, 16");
    constexpr int q = (R == 8) ? 2 * Q : Q;  // express as a 16th root
    if constexpr (q == 0) return a;
    else if constexpr (q == 4) return cmul_mi(a);
    else if constexpr (std::is_same_v<T, P2>) return rot_p2<q>(a);
    else if constexpr (q == 2) return cmulc(a, kC8, -kC8);
    else if constexpr (q == 6) return cmulc(a, -kC8, -kC8);
    else if constexpr (q == 1) return cmulc(a, kC16, -kS16);
    else if constexpr (q == 3) return cmulc(a, kS16, -kC16);
    else if constexpr (q == 5) return cmulc(a, -kS16, -kC16);
    else return cmulc(a, -kC16, -kS16);  // q == 7
}

// In-register DFT of R values, natural order in and out:
//   v[q] <- sum_r v[r] exp(-2 pi i r q / R).
// R = 8 and 16 split into even- and odd-indexed halves (decimation in time).
template <int R> struct Dft;

template <> struct Dft<1> {
    template <typename T> __device__ __forceinline__ static void run(T (&)[1]) {}
};

template <> struct Dft<2> {
    template <typename T> __device__ __forceinline__ static void run(T (&v)[2]) {
        T a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <> struct Dft<4> {
    template <typename T> __device__ __forceinline__ static void run(T (&v)[4]) {
        T a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        T c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = add_mi(b, d);  // b + (-i) d
        v[3] = sub_mi(b, d);
    }
};

template <int R> struct DftSplit {
    // outputs Q and Q + R/2 from the even and odd half-length DFTs
    template <int Q, typename T>
    __device__ __forceinline__ static void combine_one(T (&v)[R], const T (&e)[R / 2], const T (&o)[R / 2]) {
        if constexpr ((R == 8 ? 2 * Q : Q) == 4) {  // twiddle -i
            v[Q] = add_mi(e[Q], o[Q]);
            v[Q + R / 2] = sub_mi(e[Q], o[Q]);
        } else {
            const T t = twiddle_const<R, Q>(o[Q]);
            v[Q] = cadd(e[Q], t);
            v[Q + R / 2] = csub(e[Q], t);
        }
    }
    template <typename T, int... Q>
    __device__ __forceinline__ static void combine(T (&v)[R], T (&e)[R / 2], T (&o)[R / 2],
                                                   std::integer_sequence<int, Q...>) {
        (combine_one<Q>(v, e, o), ...);
    }
    template <typename T> __device__ __forceinline__ static void run(T (&v)[R]) {
        T e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; i++) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        Dft<R / 2>::run(e);
        Dft<R / 2>::run(o);
        combine(v, e, o, std::make_integer_sequence<int, R / 2>{});
    }
};

template <> struct Dft<8> {
    template <typename T> __device__ __forceinline__ static void run(T (&v)[8]) { DftSplit<8>::run(v); }
};
template <> struct Dft<16> {
    template <typename T> __device__ __forceinline__ static void run(T (&v)[16]) { DftSplit<16>::run(v); }
};

// Pass descriptor of an in-place decimation-in-frequency pass: blocks of
// length lb, radix r, m = lb / r butterflies per block, twiddles
// W_lb^(j*q) stored at tw[off + j*(r-1) + q-1].
struct Pass {
    int r;
    int m;
    int lb;
    int off;
    int lr;  // log2 r
    int lm;  // log2 m
};

}  // namespace vspec
