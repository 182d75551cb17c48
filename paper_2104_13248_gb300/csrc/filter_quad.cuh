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
// Transform: Stockham autosort passes of radix 16 first and last and 2, 4,
// 5, 8, 10 or 16 between them (N = 2^a or 5 * 2^a, the smallest such size
// >= 2 nu - 1). Every thread holds R points of one butterfly group in
// registers; each pass reads and writes shared memory once. The first pass
// reads the projections (cosine-weighted) from global memory and skips the
// zero half of its inputs; the last forward pass, the spectrum multiply and
// the first inverse pass (same radix and groups) are one register-resident
// step; the last inverse pass writes only the first nu outputs of each row.
//
// Shared memory: one float4 (re pair, im pair) per point, position
// m + m/16 within the quad's block, which keeps the 16-byte accesses of
// every pass free of bank conflicts. The raw rows are first staged at the
// start of the same buffer with cp.async.
#pragma once

#include <cuda_fp16.h>

#include "filter_quad.h"

namespace bp {
namespace fq {

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

template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<2, DIR> {
    __device__ __forceinline__ static void run(C2 *v) {
        const C2 a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    }
};

template <int DIR>
struct Dft<4, DIR> {
    __device__ __forceinline__ static void run(C2 *v) { dft4<DIR>(v[0], v[1], v[2], v[3]); }
};

template <int DIR>
struct Dft<5, DIR> {
    __device__ __forceinline__ static void run(C2 *v) { dft5<DIR>(v[0], v[1], v[2], v[3], v[4]); }
};

// X[k1 + 4 k2] = E[k1] + (-1)^k2 W8^k1 O[k1] with E, O the 4-point DFTs of
// the even and odd inputs
template <int DIR>
struct Dft<8, DIR> {
    __device__ __forceinline__ static void run(C2 *v) {
        C2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        C2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        dft4<DIR>(e0, e1, e2, e3);
        dft4<DIR>(o0, o1, o2, o3);
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
template <int DIR>
struct Dft<10, DIR> {
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
// 4-point DFTs over n2
template <int DIR>
struct Dft<16, DIR> {
    template <int N2, int K1>
    __device__ __forceinline__ static void tw(C2 *v) {
        v[N2 + 4 * K1] = crot<DIR, 16, N2 * K1>(v[N2 + 4 * K1]);
    }
    __device__ __forceinline__ static void run(C2 *v) {
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) dft4<DIR>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
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

// Twiddle product: angle of a plus angle of b.
__device__ __forceinline__ Tw tw_mul(Tw a, Tw b) {
    return {fma(a.c, b.c, mul(neg(a.s), b.s)), fma(a.s, b.c, mul(a.c, b.s))};
}

// x * exp(DIR i theta) for a twiddle (cos theta, sin theta)
template <int DIR>
__device__ __forceinline__ C2 tw_apply(C2 x, Tw w) {
    if constexpr (DIR < 0)
        return {fma(x.re, w.c, mul(x.im, w.s)), fma(x.im, w.c, mul(x.re, neg(w.s)))};
    else
        return {fma(x.re, w.c, mul(x.im, neg(w.s))), fma(x.im, w.c, mul(x.re, w.s))};
}

// Inter-pass twiddles of a Stockham pass: v[r] *= W_N^(DIR k r N / (NS R)).
// Angles for r = 1, 4, 8 come from the table; r = 2, 3 are products with
// r = 1, r = 5..7 with r = 4 and r = 9..15 with r = 8 (a few ulp). Each
// twiddle is applied as soon as it exists, so only the bases stay live.
// The table is read with plain (coherent) loads: the compiler may hoist
// read-only loads above the pass barriers, and hoisting every pass's
// twiddles to the kernel start doubled the register count.
template <int N, int R, int NS, int DIR>
__device__ __forceinline__ void apply_twiddles(C2 *v, int k, const ulonglong2 *tw4) {
    constexpr int step = N / (NS * R);
    const ulonglong2 t1 = tw4[k * step];
    const Tw w1 = {t1.x, t1.y};
    Tw w4 = w1, w8 = w1, w2 = w1, w3 = w1;
    if constexpr (R > 4) {
        const ulonglong2 t = tw4[k * 4 * step];
        w4 = {t.x, t.y};
    }
    if constexpr (R > 8) {
        const ulonglong2 t = tw4[k * 8 * step];
        w8 = {t.x, t.y};
    }
#pragma unroll
    for (int r = 1; r < (R < 8 ? R : 8); ++r) {
        Tw w;
        if (r == 1) w = w1;
        else if (r == 2) w = w2 = tw_mul(w1, w1);
        else if (r == 3) w = w3 = tw_mul(w1, w2);
        else if (r == 4) w = w4;
        else if (r == 5) w = tw_mul(w4, w1);
        else if (r == 6) w = tw_mul(w4, w2);
        else w = tw_mul(w4, w3);
        v[r] = tw_apply<DIR>(v[r], w);
        if (r + 8 < R) v[r + 8] = tw_apply<DIR>(v[r + 8], tw_mul(w8, w));
    }
    if constexpr (R > 8) v[8] = tw_apply<DIR>(v[8], w8);
}

__device__ __forceinline__ int pad(int m) { return m + (m >> 4); }

// Forward radix list: 16 first and last, the remaining factor between.
__host__ __device__ constexpr int plan_count(int N) {
    return N == 1280 || N == 2560 ? 3
         : N == 5120 || N == 10240 ? 4
         : N <= 128 ? 2
         : N <= 4096 ? (N == 256 ? 2 : 3)
         : 4;
}
__host__ __device__ constexpr int plan_radix(int N, int p) {
    return p == 0 ? 16
         : N == 1280 ? (p == 1 ? 5 : 16)
         : N == 2560 ? (p == 1 ? 10 : 16)
         : N == 5120 ? (p == 1 ? 5 : p == 2 ? 4 : 16)
         : N == 10240 ? (p == 1 ? 10 : p == 2 ? 4 : 16)
         : N <= 128 ? N / 16
         : N == 256 || N == 4096 ? 16
         : N == 8192 ? (p == 1 ? 2 : 16)
         : (p == 1 ? N / 256 : 16);   // 512, 1024, 2048: 16, 2|4|8, 16
}
__host__ __device__ constexpr int plan_ns(int N, int p) {   // product of radices before p
    return p == 0 ? 1 : plan_ns(N, p - 1) * plan_radix(N, p - 1);
}
template <int N>
struct QCfg {
    static constexpr int QPC = (N / 16 >= 128) ? 1 : (128 + N / 16 - 1) / (N / 16);   // quads per CTA
    static constexpr int NT = QPC * N / 16;                            // threads
    static constexpr int QS = N + N / 16;                              // float4 per quad
    static constexpr int SP = N / 2;                                   // staged row pitch (floats) >= nu
    static constexpr int BUF_BYTES = QPC * QS * 16;
    static constexpr int STAGE_BYTES = QPC * 4 * SP * 4;
    // raw rows are copied to the start of the transform buffer first (the
    // first pass reads them all before it writes)
    static constexpr bool STAGED = STAGE_BYTES <= 227 * 1024;
    static constexpr int SMEM = BUF_BYTES > STAGE_BYTES ? BUF_BYTES : STAGE_BYTES;
    // resident CTAs the register budget targets (about 100 registers a thread:
    // four CTAs of 160 threads for N = 2560; a few spills cost less than the
    // latency a fourth CTA hides)
    static constexpr int MINB = (65536 / (NT * 100)) > 1 ? 65536 / (NT * 100) : 1;
};

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Asynchronous copy of the raw rows of one work unit (QPC quads) into the
// staging area [4 QPC][SP]; rows past the end are skipped (and never read).
template <int N>
__device__ __forceinline__ void stage_rows(float *stage, const QArgs &a, long long row0) {
    constexpr int QPC = QCfg<N>::QPC, NT = QCfg<N>::NT, SP = QCfg<N>::SP;
    for (int rr = 0; rr < 4 * QPC; ++rr) {
        const long long row = row0 + rr;
        if (row >= a.nrows) break;
        const float *src = a.in + row * a.nu;
        float *dst = stage + rr * SP;
        if (a.in_vec)
            for (int c = threadIdx.x; c < a.nu / 4; c += NT) cp_async16(dst + 4 * c, src + 4 * c);
        else
            for (int c = threadIdx.x; c < a.nu; c += NT) cp_async4(dst + c, src + c);
    }
    cp_async_commit();
}

__device__ __forceinline__ void put(float *p, float x) { __stcs(p, x); }
__device__ __forceinline__ void put(__half *p, float x) { *p = __float2half_rn(x); }

// Outputs j + r G (r < RH) of the four rows of a quad; only m < nu are kept.
template <typename TO, int RH>
__device__ __forceinline__ void store_rows(const C2 *v, TO *out, long long r0, int j, int G,
                                           const QArgs &a) {
#pragma unroll
    for (int r = 0; r < RH; ++r) {
        const int m = j + r * G;
        if (m < a.nu) {
            float x[4];
            upk(v[r].re, x[0], x[2]);
            upk(v[r].im, x[1], x[3]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (r0 + i < a.nrows) put(out + (r0 + i) * a.nu + m, x[i]);
        }
    }
}

// One Stockham pass of radix R and stride NS over the CTA's quads.
//   MODE 0: shared -> shared
//   MODE 1: global (cosine-weighted) -> shared, first forward pass (NS = 1)
//   MODE 2: last forward pass, spectrum, first inverse pass; shared -> shared
//   MODE 3: shared -> global, last inverse pass (NS = N / R)
template <int N, int R, int NS, int DIR, int MODE>
__device__ __forceinline__ void qpass(ulonglong2 *buf, const float *stage, const QArgs &a,
                                      long long row0) {
    constexpr int QPC = QCfg<N>::QPC, NT = QCfg<N>::NT, QS = QCfg<N>::QS;
    constexpr int G = N / R;
    constexpr int NG = QPC * G;
    constexpr int GPT = (NG + NT - 1) / NT;
    const int tid = (int)threadIdx.x;
    C2 v[GPT][R];
#pragma unroll
    for (int q = 0; q < GPT; ++q) {
        const int g = q * NT + tid;
        if (NG % NT != 0 && g >= NG) continue;
        const int p = g / G, j = g - p * G;
        const int k = j % NS;
        if constexpr (MODE == 1) {
            // points j + r G; N >= 2 nu - 1 gives nu <= N / 2 = 8 G, so r >= 8 is padding
            static_assert(R == 16 && NS == 1, "first pass is radix 16");
            const long long r0 = row0 + 4 * p;
            const float sdd2 = a.sdd * a.sdd;
            float vm2[4];
            bool in[4];
            int rv = (int)(r0 % a.nv);   // detector row of r0 within its view
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                in[i] = r0 + i < a.nrows;
                const float vm = ((float)rv - a.cv) * a.dv;
                vm2[i] = vm * vm;
                rv = (rv + 1 == a.nv) ? 0 : rv + 1;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float x[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                const int m = j + r * G;
                if (r < R / 2 && m < a.nu) {
                    float um = ((float)m - a.cu) * a.du;
                    um *= um;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (in[i]) {
                            const float raw = QCfg<N>::STAGED ? stage[(4 * p + i) * QCfg<N>::SP + m]
                                                              : __ldcs(a.in + (r0 + i) * a.nu + m);
                            x[i] = raw * (a.sdd * rsqrtf(sdd2 + um + vm2[i]));
                        }
                    }
                }
                v[q][r] = {pk(x[0], x[2]), pk(x[1], x[3])};
            }
        } else {
            const ulonglong2 *src = buf + p * QS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const ulonglong2 t = src[pad(j + r * G)];
                v[q][r] = {t.x, t.y};
            }
        }
        if constexpr (NS > 1) apply_twiddles<N, R, NS, DIR>(v[q], k, a.tw4);
        Dft<R, DIR>::run(v[q]);
        if constexpr (MODE == 2) {
            static_assert(NS * R == N, "fused step is the last forward pass");
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const f2 h = reinterpret_cast<const unsigned long long *>(a.H2)[j + r * G];
                v[q][r] = {mul(v[q][r].re, h), mul(v[q][r].im, h)};
            }
            Dft<R, -DIR>::run(v[q]);
        }
    }
    if constexpr (MODE != 1 || QCfg<N>::STAGED) __syncthreads();   // every read of the pass precedes every write
#pragma unroll
    for (int q = 0; q < GPT; ++q) {
        const int g = q * NT + tid;
        if (NG % NT != 0 && g >= NG) continue;
        const int p = g / G, j = g - p * G;
        const int k = j % NS;
        if constexpr (MODE == 3) {
            static_assert(R == 16 && NS * R == N, "last pass is radix 16");
            // outputs j + r G; only m < nu <= 8 G are kept
            const long long r0 = row0 + 4 * p;
            if (a.out_f16)
                store_rows<__half, R / 2>(v[q], reinterpret_cast<__half *>(a.out), r0, j, NS, a);
            else
                store_rows<float, R / 2>(v[q], reinterpret_cast<float *>(a.out), r0, j, NS, a);
        } else {
            ulonglong2 *dst = buf + p * QS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int m = (MODE == 2) ? j * R + r : (j - k) * R + k + r * NS;
                dst[pad(m)] = make_ulonglong2(v[q][r].re, v[q][r].im);
            }
        }
    }
    if constexpr (MODE != 3) __syncthreads();
}

template <int N, int P>
__device__ __forceinline__ void forward_passes(ulonglong2 *buf, const float *stage, const QArgs &a,
                                               long long row0) {
    constexpr int C = plan_count(N);
    if constexpr (P < C) {
        constexpr int MODE = P == 0 ? 1 : (P == C - 1 ? 2 : 0);
        qpass<N, plan_radix(N, P), plan_ns(N, P), -1, MODE>(buf, stage, a, row0);
        forward_passes<N, P + 1>(buf, stage, a, row0);
    }
}

// inverse pass Q (Q = 1 .. C-1; pass 0 ran inside the fused step) uses the
// forward radix list backwards
template <int N, int Q>
__device__ __forceinline__ void inverse_passes(ulonglong2 *buf, const float *stage, const QArgs &a,
                                               long long row0) {
    constexpr int C = plan_count(N);
    if constexpr (Q < C) {
        constexpr int P = C - 1 - Q;
        constexpr int R = plan_radix(N, P);
        constexpr int NS = N / (plan_ns(N, P) * R);
        qpass<N, R, NS, +1, Q == C - 1 ? 3 : 0>(buf, stage, a, row0);
        inverse_passes<N, Q + 1>(buf, stage, a, row0);
    }
}

// One unit (QPC quads) per CTA. When the rows are staged, the CTA first
// copies its raw rows into its shared memory with cp.async, so every load of
// the unit is in flight at once without holding registers. (A persistent loop
// that prefetched the next unit spilled: the compiler kept the transform's
// loop-invariant constants live across iterations.)
template <int N>
__global__ void __launch_bounds__(QCfg<N>::NT, QCfg<N>::MINB) ramp_filter_quad(QArgs a) {
    extern __shared__ ulonglong2 qbuf[];
    using Cfg = QCfg<N>;
    float *stage = reinterpret_cast<float *>(qbuf);   // aliases the transform buffer
    const long long row0 = (long long)blockIdx.x * 4LL * Cfg::QPC;
    if constexpr (Cfg::STAGED) {
        stage_rows<N>(stage, a, row0);
        cp_async_wait_all();
        __syncthreads();
    }
    forward_passes<N, 0>(qbuf, stage, a, row0);
    inverse_passes<N, 1>(qbuf, stage, a, row0);
}

}  // namespace fq

template <int N>
cudaError_t launch_quad(const QArgs &a, cudaStream_t st) {
    using Cfg = fq::QCfg<N>;
    const long long rows_per_cta = 4LL * Cfg::QPC;
    const long long nblk = (a.nrows + rows_per_cta - 1) / rows_per_cta;
    if (nblk <= 0) return cudaSuccess;
    auto k = fq::ramp_filter_quad<N>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    if (e != cudaSuccess) return e;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidValue;
    k<<<(unsigned)nblk, Cfg::NT, Cfg::SMEM, st>>>(a);
    return cudaGetLastError();
}

}  // namespace bp
