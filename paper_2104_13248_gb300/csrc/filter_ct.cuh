// FDK pre-filter on four detector rows at a time: cosine weight, then the
// linear convolution of every row with the discrete Ram-Lak kernel as a
// zero-padded FFT convolution in shared memory (the paper assumes filtered
// projections, Section 2.1.2).
//
// Rows (4q, 4q+1) are the real and imaginary parts of one complex transform
// and rows (4q+2, 4q+3) of a second one; the kernel's spectrum is real and
// even, so the product keeps the two rows of a transform apart. The two
// transforms run side by side in packed f32x2 registers (split complex:
// re = (row 4q, row 4q+2), im = (row 4q+1, row 4q+3)), so every packed
// instruction advances four rows.
//
// Transform: in-place mixed-radix Cooley-Tukey. The forward transform
// decimates in frequency (radix R_p on sub-blocks of span S_p, stride
// T_p = S_p / R_p, twiddles after each DFT) and leaves the spectrum in
// digit-reversed order; the inverse decimates in time with the passes in
// reverse (conjugate twiddles before each DFT) and returns natural order. A
// convolution needs no reordering: the spectrum table is stored in the same
// digit-reversed order. Every butterfly group reads and writes the same
// shared-memory slots, so a pass needs no barrier between its reads and its
// writes, only one after it. The radices are 16 first and last, with the
// remaining factor (2, 4, 5, 8, 10, or 5 and 4, 10 and 4, 2 and 16) between
// (N <= 128: N / 16, then 16); every stride is 1 or a multiple of 16, so a
// group's slots are one base address plus compile-time offsets.
//
// The first pass reads the projections (cosine-weighted) from global memory
// and skips the zero half of its inputs; the last forward pass, the
// spectrum multiply and the first inverse pass (the same 16 contiguous
// points) are one register-resident step; the last pass writes only the
// first nu outputs of each row.
//
// Shared memory: one 16-byte slot (re pair, im pair) per point, position m
// at slot m + m / 16, which keeps the 16-byte accesses of every pass free of
// bank conflicts.
#pragma once

#include <cuda_fp16.h>

#include "filter_ct.h"

namespace bp {
namespace fct {

typedef unsigned long long f2;   // two FP32 lanes
struct C2 {
    f2 re, im;
};
struct Tw {
    f2 c, s;                     // cos and sin of the twiddle angle, both lanes equal
};

__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2 splat(float a) { return pk(a, a); }
__device__ __forceinline__ f2 add(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2 neg(f2 a) { return sub(0ull, a); }

__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {add(a.re, b.re), add(a.im, b.im)}; }
__device__ __forceinline__ C2 csub(C2 a, C2 b) { return {sub(a.re, b.re), sub(a.im, b.im)}; }
// a + S i b (S = +1 or -1)
template <int S>
__device__ __forceinline__ C2 add_ib(C2 a, C2 b) {
    if constexpr (S > 0)
        return {sub(a.re, b.im), add(a.im, b.re)};
    else
        return {add(a.re, b.im), sub(a.im, b.re)};
}

// cos and sin of 2 pi e / 80 (80 is a multiple of every radix used)
constexpr float kCos80[80] = {
    1.000000000f, 9.969173337e-01f, 9.876883406e-01f, 9.723699204e-01f, 9.510565163e-01f,
    9.238795325e-01f, 8.910065242e-01f, 8.526401644e-01f, 8.090169944e-01f, 7.604059656e-01f,
    7.071067812e-01f, 6.494480483e-01f, 5.877852523e-01f, 5.224985647e-01f, 4.539904997e-01f,
    3.826834324e-01f, 3.090169944e-01f, 2.334453639e-01f, 1.564344650e-01f, 7.845909573e-02f,
    6.123233996e-17f, -7.845909573e-02f, -1.564344650e-01f, -2.334453639e-01f, -3.090169944e-01f,
    -3.826834324e-01f, -4.539904997e-01f, -5.224985647e-01f, -5.877852523e-01f, -6.494480483e-01f,
    -7.071067812e-01f, -7.604059656e-01f, -8.090169944e-01f, -8.526401644e-01f, -8.910065242e-01f,
    -9.238795325e-01f, -9.510565163e-01f, -9.723699204e-01f, -9.876883406e-01f, -9.969173337e-01f,
    -1.000000000f, -9.969173337e-01f, -9.876883406e-01f, -9.723699204e-01f, -9.510565163e-01f,
    -9.238795325e-01f, -8.910065242e-01f, -8.526401644e-01f, -8.090169944e-01f, -7.604059656e-01f,
    -7.071067812e-01f, -6.494480483e-01f, -5.877852523e-01f, -5.224985647e-01f, -4.539904997e-01f,
    -3.826834324e-01f, -3.090169944e-01f, -2.334453639e-01f, -1.564344650e-01f, -7.845909573e-02f,
    -1.836970199e-16f, 7.845909573e-02f, 1.564344650e-01f, 2.334453639e-01f, 3.090169944e-01f,
    3.826834324e-01f, 4.539904997e-01f, 5.224985647e-01f, 5.877852523e-01f, 6.494480483e-01f,
    7.071067812e-01f, 7.604059656e-01f, 8.090169944e-01f, 8.526401644e-01f, 8.910065242e-01f,
    9.238795325e-01f, 9.510565163e-01f, 9.723699204e-01f, 9.876883406e-01f, 9.969173337e-01f};
constexpr float kSin80[80] = {
    0.000000000f, 7.845909573e-02f, 1.564344650e-01f, 2.334453639e-01f, 3.090169944e-01f,
    3.826834324e-01f, 4.539904997e-01f, 5.224985647e-01f, 5.877852523e-01f, 6.494480483e-01f,
    7.071067812e-01f, 7.604059656e-01f, 8.090169944e-01f, 8.526401644e-01f, 8.910065242e-01f,
    9.238795325e-01f, 9.510565163e-01f, 9.723699204e-01f, 9.876883406e-01f, 9.969173337e-01f,
    1.000000000f, 9.969173337e-01f, 9.876883406e-01f, 9.723699204e-01f, 9.510565163e-01f,
    9.238795325e-01f, 8.910065242e-01f, 8.526401644e-01f, 8.090169944e-01f, 7.604059656e-01f,
    7.071067812e-01f, 6.494480483e-01f, 5.877852523e-01f, 5.224985647e-01f, 4.539904997e-01f,
    3.826834324e-01f, 3.090169944e-01f, 2.334453639e-01f, 1.564344650e-01f, 7.845909573e-02f,
    1.224646799e-16f, -7.845909573e-02f, -1.564344650e-01f, -2.334453639e-01f, -3.090169944e-01f,
    -3.826834324e-01f, -4.539904997e-01f, -5.224985647e-01f, -5.877852523e-01f, -6.494480483e-01f,
    -7.071067812e-01f, -7.604059656e-01f, -8.090169944e-01f, -8.526401644e-01f, -8.910065242e-01f,
    -9.238795325e-01f, -9.510565163e-01f, -9.723699204e-01f, -9.876883406e-01f, -9.969173337e-01f,
    -1.000000000f, -9.969173337e-01f, -9.876883406e-01f, -9.723699204e-01f, -9.510565163e-01f,
    -9.238795325e-01f, -8.910065242e-01f, -8.526401644e-01f, -8.090169944e-01f, -7.604059656e-01f,
    -7.071067812e-01f, -6.494480483e-01f, -5.877852523e-01f, -5.224985647e-01f, -4.539904997e-01f,
    -3.826834324e-01f, -3.090169944e-01f, -2.334453639e-01f, -1.564344650e-01f, -7.845909573e-02f};

// x * exp(DIR * 2 pi i * m / M) for compile-time m, M (M divides 80)
template <int DIR, int M, int m>
__device__ __forceinline__ C2 crot(C2 x) {
    constexpr int e = ((m % M) + M) % M * (80 / M);
    if constexpr (e == 0) {
        return x;
    } else if constexpr (e == 40) {
        return {neg(x.re), neg(x.im)};
    } else if constexpr (e == 20 || e == 60) {
        // multiply by S i with S = DIR for a quarter turn, -DIR for three quarters
        constexpr int S = (e == 20) ? DIR : -DIR;
        if constexpr (S > 0)
            return {neg(x.im), x.re};
        else
            return {x.im, neg(x.re)};
    } else {
        const float c = kCos80[e], s = DIR * kSin80[e];
        return {fma(x.re, splat(c), mul(x.im, splat(-s))), fma(x.im, splat(c), mul(x.re, splat(s)))};
    }
}

template <int DIR>
__device__ __forceinline__ void dft4(C2 &x0, C2 &x1, C2 &x2, C2 &x3) {
    const C2 a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), e = csub(x1, x3);
    x0 = cadd(a, c);
    x2 = csub(a, c);
    x1 = add_ib<DIR>(b, e);
    x3 = add_ib<-DIR>(b, e);
}

// dft4 of (x0, x1, 0, 0)
template <int DIR>
__device__ __forceinline__ void dft4_half(C2 &x0, C2 &x1, C2 &x2, C2 &x3) {
    const C2 a = x0, b = x1;
    x0 = cadd(a, b);
    x2 = csub(a, b);
    x1 = add_ib<DIR>(a, b);
    x3 = add_ib<-DIR>(a, b);
}

// 5-point DFT: with a1 = x1 + x4, b1 = x1 - x4, a2 = x2 + x3, b2 = x2 - x3,
// X1,4 = x0 + c1 a1 + c2 a2 +- DIR i (s1 b1 + s2 b2) and
// X2,3 = x0 + c2 a1 + c1 a2 +- DIR i (s2 b1 - s1 b2), c/s of 2 pi / 5 and 4 pi / 5
template <int DIR>
__device__ __forceinline__ void dft5(C2 &x0, C2 &x1, C2 &x2, C2 &x3, C2 &x4) {
    const f2 c1 = splat(kCos80[16]), c2 = splat(kCos80[32]);
    const f2 s1 = splat(kSin80[16]), s2 = splat(kSin80[32]), ns1 = splat(-kSin80[16]);
    const C2 a1 = cadd(x1, x4), b1 = csub(x1, x4), a2 = cadd(x2, x3), b2 = csub(x2, x3);
    const C2 t1 = {fma(c2, a2.re, fma(c1, a1.re, x0.re)), fma(c2, a2.im, fma(c1, a1.im, x0.im))};
    const C2 t2 = {fma(c1, a2.re, fma(c2, a1.re, x0.re)), fma(c1, a2.im, fma(c2, a1.im, x0.im))};
    const C2 u1 = {fma(s2, b2.re, mul(s1, b1.re)), fma(s2, b2.im, mul(s1, b1.im))};
    const C2 u2 = {fma(ns1, b2.re, mul(s2, b1.re)), fma(ns1, b2.im, mul(s2, b1.im))};
    x0 = cadd(x0, cadd(a1, a2));
    x1 = add_ib<DIR>(t1, u1);
    x4 = add_ib<-DIR>(t1, u1);
    x2 = add_ib<DIR>(t2, u2);
    x3 = add_ib<-DIR>(t2, u2);
}

// R-point DFTs in registers, X[k] = sum_n x[n] exp(DIR 2 pi i n k / R), in
// natural order in and out. HALF: inputs n >= R / 2 are zero (not read).
template <int R, int DIR, bool HALF = false>
struct Dft;

template <int DIR, bool HALF>
struct Dft<2, DIR, HALF> {
    __device__ __forceinline__ static void run(C2 *v) {
        if constexpr (HALF) {
            v[1] = v[0];
        } else {
            const C2 a = v[0];
            v[0] = cadd(a, v[1]);
            v[1] = csub(a, v[1]);
        }
    }
};

template <int DIR, bool HALF>
struct Dft<4, DIR, HALF> {
    __device__ __forceinline__ static void run(C2 *v) {
        if constexpr (HALF)
            dft4_half<DIR>(v[0], v[1], v[2], v[3]);
        else
            dft4<DIR>(v[0], v[1], v[2], v[3]);
    }
};

template <int DIR, bool HALF>
struct Dft<5, DIR, HALF> {
    static_assert(!HALF, "radix 5 is never a first pass");
    __device__ __forceinline__ static void run(C2 *v) { dft5<DIR>(v[0], v[1], v[2], v[3], v[4]); }
};

// X[k1 + 4 k2] = E[k1] + (-1)^k2 W8^k1 O[k1] with E, O the 4-point DFTs of
// the even and odd inputs
template <int DIR, bool HALF>
struct Dft<8, DIR, HALF> {
    __device__ __forceinline__ static void run(C2 *v) {
        C2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        C2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        if constexpr (HALF) {
            dft4_half<DIR>(e0, e1, e2, e3);
            dft4_half<DIR>(o0, o1, o2, o3);
        } else {
            dft4<DIR>(e0, e1, e2, e3);
            dft4<DIR>(o0, o1, o2, o3);
        }
        o1 = crot<DIR, 8, 1>(o1);
        o3 = crot<DIR, 8, 3>(o3);
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
        v[2] = add_ib<DIR>(e2, o2); v[6] = add_ib<-DIR>(e2, o2);   // W8^2 = DIR i
        v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
    }
};

// X[k1 + 5 k2] = E[k1] + (-1)^k2 W10^k1 O[k1] with E, O the 5-point DFTs of
// the even and odd inputs
template <int DIR, bool HALF>
struct Dft<10, DIR, HALF> {
    static_assert(!HALF, "radix 10 is never a first pass");
    __device__ __forceinline__ static void run(C2 *v) {
        C2 e[5] = {v[0], v[2], v[4], v[6], v[8]};
        C2 o[5] = {v[1], v[3], v[5], v[7], v[9]};
        dft5<DIR>(e[0], e[1], e[2], e[3], e[4]);
        dft5<DIR>(o[0], o[1], o[2], o[3], o[4]);
        o[1] = crot<DIR, 10, 1>(o[1]);
        o[2] = crot<DIR, 10, 2>(o[2]);
        o[3] = crot<DIR, 10, 3>(o[3]);
        o[4] = crot<DIR, 10, 4>(o[4]);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 5] = csub(e[k], o[k]);
        }
    }
};

// n = 4 n1 + n2, k = k1 + 4 k2: 4-point DFTs over n1, twiddles W16^(n2 k1),
// 4-point DFTs over n2 (HALF: n1 >= 2 are the zero inputs)
template <int DIR, bool HALF>
struct Dft<16, DIR, HALF> {
    template <int N2, int K1>
    __device__ __forceinline__ static void tw(C2 *v) {
        v[N2 + 4 * K1] = crot<DIR, 16, N2 * K1>(v[N2 + 4 * K1]);
    }
    __device__ __forceinline__ static void run(C2 *v) {
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            if constexpr (HALF)
                dft4_half<DIR>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
            else
                dft4<DIR>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
        }
        // v[n2 + 4 k1] now holds A[n2][k1]
        tw<1, 1>(v); tw<1, 2>(v); tw<1, 3>(v);
        tw<2, 1>(v); tw<2, 2>(v); tw<2, 3>(v);
        tw<3, 1>(v); tw<3, 2>(v); tw<3, 3>(v);
        C2 t[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C2 a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
            dft4<DIR>(a0, a1, a2, a3);
            t[k1] = a0; t[k1 + 4] = a1; t[k1 + 8] = a2; t[k1 + 12] = a3;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = t[i];
    }
};

// x * exp(DIR i theta) for a twiddle (cos theta, sin theta)
template <int DIR>
__device__ __forceinline__ C2 tw_apply(C2 x, Tw w) {
    if constexpr (DIR < 0)
        return {fma(x.re, w.c, mul(x.im, w.s)), fma(x.im, w.c, mul(x.re, neg(w.s)))};
    else
        return {fma(x.re, w.c, mul(x.im, neg(w.s))), fma(x.im, w.c, mul(x.re, w.s))};
}

// ---- plan -----------------------------------------------------------------

// Number of passes and their radices; the last radix is 16 (the fused step
// works on 16 contiguous points).
__host__ __device__ constexpr int plan_count(int N) {
    return N <= 256 ? 2 : (N == 5120 || N == 8192 || N == 10240) ? 4 : 3;
}
__host__ __device__ constexpr int plan_radix(int N, int p) {
    return N <= 128 ? (p == 0 ? N / 16 : 16)
         : N == 256 ? 16
         : N == 8192 ? (p == 1 ? 2 : 16)
         : N == 5120 ? (p == 1 ? 5 : p == 2 ? 4 : 16)
         : N == 10240 ? (p == 1 ? 10 : p == 2 ? 4 : 16)
         : (p == 1 ? N / 256 : 16);   // 512 .. 4096, 1280, 2560
}
// span S_p of pass p's sub-blocks and stride T_p = S_p / R_p of a group's points
__host__ __device__ constexpr int plan_span(int N, int p) {
    return p == 0 ? N : plan_span(N, p - 1) / plan_radix(N, p - 1);
}
__host__ __device__ constexpr int plan_stride(int N, int p) { return plan_span(N, p) / plan_radix(N, p); }
// first twiddle-table entry of pass p: entries (k - 1) T_p + o for k in [1, R_p), o in [0, T_p)
__host__ __device__ constexpr int plan_tw_offset(int N, int p) {
    return p == 0 ? 0 : plan_tw_offset(N, p - 1) + (plan_radix(N, p - 1) - 1) * plan_stride(N, p - 1);
}

template <int N>
struct Cfg {
    static constexpr int C = plan_count(N);
    static constexpr int QPC = (N / 16 >= 128) ? 1 : (128 + N / 16 - 1) / (N / 16);   // quads per CTA
    static constexpr int NT = QPC * N / 16;                            // threads
    static constexpr int QS = N + N / 16;                              // 16-byte slots per quad
    static constexpr int SMEM = QPC * QS * 16;
    // resident CTAs the register budget targets (about 100 registers a
    // thread: four CTAs of 160 threads for N = 2560; 80 registers and five
    // CTAs spilled and ran slower)
    static constexpr int MINB = (65536 / (NT * 100)) > 1 ? 65536 / (NT * 100) : 1;
};

// Pass p's butterfly groups: NG over the CTA's quads, GPT per thread, taken
// by the first ACT threads (g = tid + q ACT): a radix-10 or radix-5 pass has
// 1.6 or 3.2 groups per thread, so a fifth of the threads sit it out and
// every warp stays convergent.
template <int N, int P>
struct Pass {
    static constexpr int R = plan_radix(N, P), S = plan_span(N, P), T = S / R;
    static constexpr int GQ = N / R;                       // groups per quad
    static constexpr int NG = Cfg<N>::QPC * GQ;
    static constexpr int GPT = (NG + Cfg<N>::NT - 1) / Cfg<N>::NT;
    static constexpr int ACT = NG / GPT;
    static constexpr int STEP = (T == 1) ? 1 : T + T / 16;   // slots between a group's points
    static constexpr int TWO = plan_tw_offset(N, P);
    static_assert(NG % GPT == 0 && ACT <= Cfg<N>::NT && ACT % 32 == 0, "groups per thread");
    static_assert(T == 1 || T % 16 == 0, "strides are 1 or multiples of 16");
    // slot of the group's first point (quad-relative) and its offset o in the sub-block
    __device__ __forceinline__ static int slot(int gl, int &o) {
        const int b = gl / T;
        o = gl - b * T;
        if constexpr (T == 1)
            return 17 * b;                  // S = 16: positions 16 b + n
        else
            return b * (S + S / 16) + o + (o >> 4);
    }
};

// ---- twiddles ---------------------------------------------------------------

// Product of twiddle a (with nsa = -a.s) and b.
__device__ __forceinline__ Tw tw_mulns(Tw a, f2 nsa, Tw b) {
    return {fma(a.c, b.c, mul(nsa, b.s)), fma(a.s, b.c, mul(a.c, b.s))};
}
__device__ __forceinline__ Tw tw_ld(const ulonglong2 *p) {
    const ulonglong2 t = *p;
    return {t.x, t.y};
}

// v[k] *= exp(DIR 2 pi i o k / S) for k = 1 .. R-1, tw = the pass's table at o
// (entry (k - 1) T). Radix 16 reads the angles of k = 1, 2, 3, 4, 8, 12 and
// forms the others as one product k = b + j (b = 4, 8, 12, j = 1, 2, 3; a
// few ulp); smaller radices read every angle (their tables are small).
template <int R, int T, int DIR>
__device__ __forceinline__ void twiddle(C2 *v, const ulonglong2 *tw) {
    if constexpr (R == 16) {
        const Tw w1 = tw_ld(tw), w2 = tw_ld(tw + T), w3 = tw_ld(tw + 2 * T);
        v[1] = tw_apply<DIR>(v[1], w1);
        v[2] = tw_apply<DIR>(v[2], w2);
        v[3] = tw_apply<DIR>(v[3], w3);
#pragma unroll
        for (int b = 4; b < 16; b += 4) {
            const Tw wb = tw_ld(tw + (b - 1) * T);
            const f2 nsb = neg(wb.s);
            v[b] = tw_apply<DIR>(v[b], wb);
            v[b + 1] = tw_apply<DIR>(v[b + 1], tw_mulns(wb, nsb, w1));
            v[b + 2] = tw_apply<DIR>(v[b + 2], tw_mulns(wb, nsb, w2));
            v[b + 3] = tw_apply<DIR>(v[b + 3], tw_mulns(wb, nsb, w3));
        }
    } else {
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = tw_apply<DIR>(v[k], tw_ld(tw + (k - 1) * T));
    }
}

// ---- first and last pass helpers ------------------------------------------

// 1 / sqrt(x) for the cosine weight (x >= sdd^2, far from denormals)
__device__ __forceinline__ float rsqrt_fast(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void put(float *p, float x) { __stcs(p, x); }
__device__ __forceinline__ void put(__half *p, float x) { *p = __float2half_rn(x); }

// ---- passes -----------------------------------------------------------------

// First pass (p = 0, forward): raw rows times the cosine weight
// rsqrt(sdd^2 + u^2 + v^2) (its factor sdd is in the spectrum), the DFT of
// the nonzero half, twiddles, and the results go to the transform slots.
// Every thread loads its points straight from global memory (consecutive
// lanes read consecutive pixels), all of them before any arithmetic; points
// past nu and rows past the end read as zeros.
template <int N>
__device__ __forceinline__ void pass_first(ulonglong2 *buf, const CtArgs &a, long long row0) {
    using PS = Pass<N, 0>;
    constexpr int R = PS::R, T = PS::T, GPT = PS::GPT, ACT = PS::ACT;
    constexpr int QS = Cfg<N>::QS;
    static_assert(T * (R / 2) == N / 2, "the first pass reads the first N / 2 points");
    const int tid = (int)threadIdx.x;
    C2 v[GPT][R];
    int sl[GPT];
    if (tid < ACT) {
#pragma unroll
        for (int q = 0; q < GPT; ++q) {
            const int g = tid + q * ACT;
            const int qd = g / PS::GQ, gl = g - qd * PS::GQ;
            int o;
            sl[q] = qd * QS + PS::slot(gl, o);
            // rows 4 qd + i: (sdd^2 + v^2) as (row 0, row 2) and (row 1, row 3)
            const long long r0 = row0 + 4 * qd;
            int rv = (int)((unsigned)r0 % (unsigned)a.nv);   // rows < 2^32 (each holds nu >= 16 floats)
            float A[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float vm = ((float)rv - a.cv) * a.dv;
                A[i] = fmaf(vm, vm, a.sdd2);
                rv = (rv + 1 == a.nv) ? 0 : rv + 1;
            }
            const f2 Are = pk(A[0], A[2]), Aim = pk(A[1], A[3]);
            const int nr = (int)min(4LL, a.nrows - r0);
            const float *s0 = a.in + r0 * a.nu + o;
            float xr[R / 2][4];
#pragma unroll
            for (int n = 0; n < R / 2; ++n)
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    xr[n][i] = (i < nr && o + n * T < a.nu) ? __ldcs(s0 + (long long)i * a.nu + n * T) : 0.0f;
            f2 UM = splat(((float)o - a.cu) * a.du);
            const f2 DU = splat((float)T * a.du);
#pragma unroll
            for (int n = 0; n < R / 2; ++n) {
                const f2 U2 = mul(UM, UM);
                float d0, d1, d2, d3;
                upk(add(Are, U2), d0, d2);
                upk(add(Aim, U2), d1, d3);
                const f2 Wre = pk(rsqrt_fast(d0), rsqrt_fast(d2)), Wim = pk(rsqrt_fast(d1), rsqrt_fast(d3));
                const f2 Xre = pk(xr[n][0], xr[n][2]);
                const f2 Xim = pk(xr[n][1], xr[n][3]);
                v[q][n] = {mul(Xre, Wre), mul(Xim, Wim)};
                UM = add(UM, DU);
            }
#pragma unroll
            for (int n = R / 2; n < R; ++n) v[q][n] = {0ull, 0ull};   // never read by the half DFT
            Dft<R, -1, true>::run(v[q]);
            if constexpr (T > 1) twiddle<R, T, -1>(v[q], a.tw + PS::TWO + o);
        }
    }
    if (tid < ACT) {
#pragma unroll
        for (int q = 0; q < GPT; ++q) {
            ulonglong2 *d = buf + sl[q];
#pragma unroll
            for (int n = 0; n < R; ++n) d[n * PS::STEP] = make_ulonglong2(v[q][n].re, v[q][n].im);
        }
    }
    __syncthreads();
}

// Middle pass p, forward (DIR = -1: DFT, then twiddles) or inverse
// (DIR = +1: conjugate twiddles, then DFT), in place.
template <int N, int P, int DIR>
__device__ __forceinline__ void pass_mid(ulonglong2 *buf, const CtArgs &a) {
    using PS = Pass<N, P>;
    constexpr int R = PS::R, T = PS::T;
    const int tid = (int)threadIdx.x;
    if (tid < PS::ACT) {
#pragma unroll
        for (int q = 0; q < PS::GPT; ++q) {
            const int g = tid + q * PS::ACT;
            const int qd = g / PS::GQ, gl = g - qd * PS::GQ;
            int o;
            ulonglong2 *d = buf + qd * Cfg<N>::QS + PS::slot(gl, o);
            C2 v[R];
#pragma unroll
            for (int n = 0; n < R; ++n) {
                const ulonglong2 t = d[n * PS::STEP];
                v[n] = {t.x, t.y};
            }
            if constexpr (DIR > 0) twiddle<R, T, +1>(v, a.tw + PS::TWO + o);
            Dft<R, DIR>::run(v);
            if constexpr (DIR < 0) twiddle<R, T, -1>(v, a.tw + PS::TWO + o);
#pragma unroll
            for (int n = 0; n < R; ++n) d[n * PS::STEP] = make_ulonglong2(v[n].re, v[n].im);
        }
    }
    __syncthreads();
}

// Fused step (p = C - 1, radix 16, 16 contiguous points): forward DFT,
// spectrum multiply, inverse DFT, in place.
template <int N>
__device__ __forceinline__ void pass_fused(ulonglong2 *buf, const CtArgs &a) {
    using PS = Pass<N, Cfg<N>::C - 1>;
    static_assert(PS::R == 16 && PS::T == 1 && PS::GPT == 1, "fused step");
    const int g = (int)threadIdx.x;
    const int qd = g / PS::GQ, gl = g - qd * PS::GQ;
    int o;
    ulonglong2 *d = buf + qd * Cfg<N>::QS + PS::slot(gl, o);
    const f2 *h = reinterpret_cast<const f2 *>(a.Ht) + gl;
    C2 v[16];
#pragma unroll
    for (int n = 0; n < 16; ++n) {
        const ulonglong2 t = d[n];
        v[n] = {t.x, t.y};
    }
    Dft<16, -1>::run(v);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const f2 hk = h[k * PS::GQ];
        v[k] = {mul(v[k].re, hk), mul(v[k].im, hk)};
    }
    Dft<16, +1>::run(v);
#pragma unroll
    for (int n = 0; n < 16; ++n) d[n] = make_ulonglong2(v[n].re, v[n].im);
    __syncthreads();
}

// Last pass (p = 0, inverse): conjugate twiddles, DFT, and the outputs
// o + n T (n < R / 2, only those below nu) of the quad's four rows go to
// global memory.
template <int N, typename TO>
__device__ __forceinline__ void pass_last(const ulonglong2 *buf, const CtArgs &a, long long row0) {
    using PS = Pass<N, 0>;
    constexpr int R = PS::R, T = PS::T;
    const int tid = (int)threadIdx.x;
    if (tid >= PS::ACT) return;
    TO *out = reinterpret_cast<TO *>(a.out);
#pragma unroll
    for (int q = 0; q < PS::GPT; ++q) {
        const int g = tid + q * PS::ACT;
        const int qd = g / PS::GQ, gl = g - qd * PS::GQ;
        int o;
        const ulonglong2 *d = buf + qd * Cfg<N>::QS + PS::slot(gl, o);
        C2 v[R];
#pragma unroll
        for (int n = 0; n < R; ++n) {
            const ulonglong2 t = d[n * PS::STEP];
            v[n] = {t.x, t.y};
        }
        if constexpr (T > 1) twiddle<R, T, +1>(v, a.tw + PS::TWO + o);
        Dft<R, +1>::run(v);
        const long long r0 = row0 + 4 * qd;
        const int nr = (int)min(4LL, a.nrows - r0);   // rows of the quad that exist
        TO *o0 = out + r0 * a.nu + o;
#pragma unroll
        for (int n = 0; n < R / 2; ++n) {
            if (o + n * T < a.nu) {
                float x[4];
                upk(v[n].re, x[0], x[2]);
                upk(v[n].im, x[1], x[3]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (i < nr) put(o0 + (long long)i * a.nu + n * T, x[i]);
            }
        }
    }
}

template <int N, int P>
__device__ __forceinline__ void forward_mids(ulonglong2 *buf, const CtArgs &a) {
    if constexpr (P < Cfg<N>::C - 1) {
        pass_mid<N, P, -1>(buf, a);
        forward_mids<N, P + 1>(buf, a);
    }
}
template <int N, int P>
__device__ __forceinline__ void inverse_mids(ulonglong2 *buf, const CtArgs &a) {
    if constexpr (P >= 1) {
        pass_mid<N, P, +1>(buf, a);
        inverse_mids<N, P - 1>(buf, a);
    }
}

// One unit (QPC quads) per CTA; four barriers in all (one after each pass
// but the last).
template <int N>
__global__ void __launch_bounds__(Cfg<N>::NT, Cfg<N>::MINB) ramp_filter_ct(CtArgs a) {
    extern __shared__ __align__(16) ulonglong2 cbuf[];
    const long long row0 = (long long)blockIdx.x * 4LL * Cfg<N>::QPC;
    pass_first<N>(cbuf, a, row0);
    forward_mids<N, 1>(cbuf, a);
    pass_fused<N>(cbuf, a);
    inverse_mids<N, Cfg<N>::C - 2>(cbuf, a);
    if (a.out_f16)
        pass_last<N, __half>(cbuf, a, row0);
    else
        pass_last<N, float>(cbuf, a, row0);
}

}  // namespace fct

template <int N>
cudaError_t launch_ct(const CtArgs &a, cudaStream_t st) {
    using Cfg = fct::Cfg<N>;
    const long long rows_per_cta = 4LL * Cfg::QPC;
    const long long nblk = (a.nrows + rows_per_cta - 1) / rows_per_cta;
    if (nblk <= 0) return cudaSuccess;
    auto k = fct::ramp_filter_ct<N>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    if (e != cudaSuccess) return e;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidValue;
    k<<<(unsigned)nblk, Cfg::NT, Cfg::SMEM, st>>>(a);
    return cudaGetLastError();
}

}  // namespace bp
