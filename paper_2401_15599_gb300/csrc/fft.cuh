// Device FFT building blocks for the multislice passes.
//
// A length-N transform is done by TPT = N / E cooperating threads, each
// holding E complex values in registers.  The algorithm is the Stockham
// autosort formulation: for stage l with radix R and NS = R_1 ... R_{l-1},
// butterfly j (0 <= j < N/R) reads positions j + r N/R, multiplies input r by
// W_{NS R}^{(j mod NS) r}, applies an R-point DFT and writes output r to
// position (j / NS) NS R + (j mod NS) + r NS.  Thread t owns butterflies
// j = t + b TPT, b = 0 .. E/R - 1.  Values move between stages through
// shared memory (two buffers, one barrier per exchange).
//
// At the boundaries (first-stage input, last-stage output) thread t holds
// positions t + TPT m, m = 0 .. E-1, in register m ("canonical order"), so
// global loads and stores are coalesced across threads and point-wise
// multiplications (transmission, propagator) can be applied in registers
// between an inverse and a forward transform without any exchange.
//
// Twiddles come from per-stage tables computed in FP64 and rounded once to
// float: for every stage with NS > 1 the block tw[OFF + (r-1) NS + jm] holds
// W_{NS R}^{jm r} (r = 1 .. R-1, jm = 0 .. NS-1), so lanes with consecutive
// jm read consecutive entries (or the same entry) of shared memory.  The
// inverse transform uses their conjugates and is unnormalised.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace tacaw {
namespace fft {

// ---------------------------------------------------------------- small DFTs
__device__ __forceinline__ float2 mul_neg_i(float2 a) { return make_float2(a.y, -a.x); }
__device__ __forceinline__ float2 mul_pos_i(float2 a) { return make_float2(-a.y, a.x); }

template <bool INV>
__device__ __forceinline__ float2 rot4(float2 a) {  // multiply by W_4 = -i (forward) / +i (inverse)
    return INV ? mul_pos_i(a) : mul_neg_i(a);
}

template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2* x) {
        float2 a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};

template <bool INV>
struct Dft<3, INV> {
    __device__ __forceinline__ static void run(float2* x) {
        const float h = 0.8660254037844386f;  // sqrt(3)/2
        float2 t1 = cadd(x[1], x[2]);
        float2 t2 = csub(x[1], x[2]);
        float2 m = make_float2(x[0].x - 0.5f * t1.x, x[0].y - 0.5f * t1.y);
        // forward: W_3 = -1/2 - i sqrt(3)/2 ; the i sqrt(3)/2 t2 term takes the sign
        float2 r = INV ? mul_pos_i(t2) : mul_neg_i(t2);
        r = cscale(r, h);
        x[0] = cadd(x[0], t1);
        x[1] = cadd(m, r);
        x[2] = csub(m, r);
    }
};

template <bool INV>
struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2* x) {
        float2 t0 = cadd(x[0], x[2]), t1 = csub(x[0], x[2]);
        float2 t2 = cadd(x[1], x[3]), t3 = rot4<INV>(csub(x[1], x[3]));
        x[0] = cadd(t0, t2);
        x[2] = csub(t0, t2);
        x[1] = cadd(t1, t3);
        x[3] = csub(t1, t3);
    }
};

template <bool INV>
struct Dft<8, INV> {
    // y[k] = E[k] + W8^k O[k], y[k+4] = E[k] - W8^k O[k] with E, O the
    // 4-point DFTs of the even and odd inputs.
    __device__ __forceinline__ static void run(float2* x) {
        const float c = 0.70710678118654752f;
        float2 e[4] = {x[0], x[2], x[4], x[6]};
        float2 o[4] = {x[1], x[3], x[5], x[7]};
        Dft<4, INV>::run(e);
        Dft<4, INV>::run(o);
        float2 o1, o2, o3;
        if (!INV) {
            o1 = make_float2((o[1].x + o[1].y) * c, (o[1].y - o[1].x) * c);   // * (1 - i)/sqrt2
            o2 = mul_neg_i(o[2]);                                            // * -i
            o3 = make_float2((o[3].y - o[3].x) * c, -(o[3].x + o[3].y) * c);  // * (-1 - i)/sqrt2
        } else {
            o1 = make_float2((o[1].x - o[1].y) * c, (o[1].x + o[1].y) * c);   // * (1 + i)/sqrt2
            o2 = mul_pos_i(o[2]);                                            // * +i
            o3 = make_float2(-(o[3].x + o[3].y) * c, (o[3].x - o[3].y) * c);  // * (-1 + i)/sqrt2
        }
        x[0] = cadd(e[0], o[0]);
        x[4] = csub(e[0], o[0]);
        x[1] = cadd(e[1], o1);
        x[5] = csub(e[1], o1);
        x[2] = cadd(e[2], o2);
        x[6] = csub(e[2], o2);
        x[3] = cadd(e[3], o3);
        x[7] = csub(e[3], o3);
    }
};

// ---------------------------------------------------------------- plans
template <int... Rs>
struct Radices {};

template <int N>
struct Plan;
template <>
struct Plan<64> { static constexpr int E = 8; using R = Radices<8, 8>; };
template <>
struct Plan<128> { static constexpr int E = 8; using R = Radices<8, 4, 4>; };
template <>
struct Plan<256> { static constexpr int E = 8; using R = Radices<8, 8, 4>; };
template <>
struct Plan<512> { static constexpr int E = 8; using R = Radices<8, 8, 8>; };
template <>
struct Plan<1024> { static constexpr int E = 8; using R = Radices<8, 8, 4, 4>; };
// long transforms (time axis): 16 values per thread
template <>
struct Plan<2048> { static constexpr int E = 16; using R = Radices<8, 8, 8, 4>; };
template <>
struct Plan<4096> { static constexpr int E = 16; using R = Radices<8, 8, 8, 8>; };
// radix-3 sizes: 24 values per thread so that every radix divides E
template <>
struct Plan<384> { static constexpr int E = 24; using R = Radices<8, 8, 2, 3>; };
template <>
struct Plan<768> { static constexpr int E = 24; using R = Radices<8, 8, 4, 3>; };

// Warp-per-row plans: one transform held by the 32 lanes of one warp, so
// every exchange needs only __syncwarp.  512 points = 16 values per thread,
// three radix-8 stages (two butterflies per thread per stage).
template <int N>
struct WarpPlan;
template <>
struct WarpPlan<512> {
    static constexpr int E = 16;
    using R = Radices<8, 8, 8>;
    static constexpr bool kDeriveTw = true;   // last stage: second butterfly's twiddles derived (see stage)
};

template <int A, int... Rest>
struct First { static constexpr int value = A; };

// Shared-memory layouts.  (Passing the same buffer as b0 and b1 to transform
// runs it in one buffer with an extra barrier per exchange.)  RowLayout: one
// transform per row, positions swizzled inside the row to spread 8-byte
// accesses over the banks.  ColLayout: W transforms interleaved
// (position-major), lanes of a warp on adjacent transforms.
struct RowLayout {
    int base;  // row * N
    __device__ __forceinline__ int operator()(int p) const { return base + (p ^ ((p >> 4) & 15)); }
};
// ColLayout: a position row of W float2 covers 2W of the 32 banks, so 16/W rows
// share the banks; the first exchange writes positions 8j + r, whose low bits
// are the same for every lane, so the position is XORed with (p >> 3) in its
// low log2(16/W) bits to spread those lanes over all bank groups.
template <int W>
struct ColLayout {
    int c;
    static constexpr int kGroups = 16 / W > 1 ? 16 / W : 1;
    __device__ __forceinline__ int operator()(int p) const { return (p ^ ((p >> 3) & (kGroups - 1))) * W + c; }
};

// Padded layouts: position p is stored at a padded index F(p), so that a
// butterfly whose positions are base + o (o compile-time offsets) computes
// F(base) once and reaches its values at F(base) + F(o): F must not carry
// between base and o, which each policy states as a condition checked below
// for the exchanges it serves.  Policies:
//   Pad16:   p + p / 16      (one spare slot after every 16; no carry when
//            (base mod 16) + (o mod 16) < 16)
//   Pad8:    p + p / 8       (no carry when (base mod 8) + (o mod 8) < 8)
//   Pad64x8: p + 8 (p / 64)  (eight spare slots after every 64; no carry when
//            (base mod 64) + (o mod 64) < 64)
// A layout takes one policy for the exchange after the first stage and one for
// the exchanges after it.  Shared memory serves a warp's 8-byte request per
// half-warp: 16 lanes in one wavefront when they reach 16 distinct bank pairs.
// Pad16 everywhere gives that for most exchanges, but not for the writes after
// the second stage of a row (lanes t and t + 8 of a half-warp collide, in every
// plan here) nor for the writes after the first stage of four or eight
// interleaved columns (lanes t and t + 1).  PadRowL<Pad16, Pad64x8> and
// PadColL<W, Pad8, Pad16> remove those where they are used: the one-warp-per-
// row pass and the staged column pass at 512 points, and the work queue's
// tiles of the 24-value plans (every exchange at the minimum, checked by
// enumerating the lanes' addresses on the host).
struct Pad16 {
    static constexpr int kRun = 16;
    __host__ __device__ static constexpr int map(int p) { return p + (p >> 4); }
    __host__ __device__ static constexpr int size(int n) { return n + n / 16; }
};
struct Pad8 {
    static constexpr int kRun = 8;
    __host__ __device__ static constexpr int map(int p) { return p + (p >> 3); }
    __host__ __device__ static constexpr int size(int n) { return n + n / 8; }
};
struct Pad64x8 {
    static constexpr int kRun = 64;
    __host__ __device__ static constexpr int map(int p) { return p + 8 * (p >> 6); }
    __host__ __device__ static constexpr int size(int n) { return n + 8 * (n / 64); }
};

template <int N>
struct PaddedLen { static constexpr int value = N + N / 16; };

__host__ __device__ constexpr int pad16(int p) { return p + (p >> 4); }

// X: exchange index (0 after the first stage).
template <class F0, class F1>
struct PadRowL {
    static constexpr bool kPadded = true;
    template <int X>
    using Pad = typename std::conditional<X == 0, F0, F1>::type;
    template <int N>
    __host__ __device__ static constexpr int slot() { return F0::size(N) > F1::size(N) ? F0::size(N) : F1::size(N); }
    int base;  // row * slot
    template <class F>
    __device__ __forceinline__ int at(int pb, int o) const { return base + pb + F::map(o); }   // pb = F(b)
};
template <int W, class F0, class F1>
struct PadColL {
    static constexpr bool kPadded = true;
    template <int X>
    using Pad = typename std::conditional<X == 0, F0, F1>::type;
    template <int N>
    __host__ __device__ static constexpr int slot() { return F0::size(N) > F1::size(N) ? F0::size(N) : F1::size(N); }
    int c;
    template <class F>
    __device__ __forceinline__ int at(int pb, int o) const { return (pb + F::map(o)) * W + c; }
};
using PadRowLayout = PadRowL<Pad16, Pad16>;
template <int W>
using PadColLayout = PadColL<W, Pad16, Pad16>;
// The layouts without half-warp collisions (see above).
using PadRowLayout512 = PadRowL<Pad16, Pad64x8>;
template <int W>
using PadColLayout512 = PadColL<W, Pad8, Pad16>;

template <class L, class = void>
struct IsPadded { static constexpr bool value = false; };
template <class L>
struct IsPadded<L, decltype(void(L::kPadded))> { static constexpr bool value = L::kPadded; };

// Twiddles of one stage (the one with NS_ = NS) held in registers by a thread
// whose butterflies there all have the same jm (one butterfly, or TPT a
// multiple of NS): w[r - 1] = W_{NS R}^{jm r}, the table's entries for its jm,
// loaded once (load_reg_tw) by a persistent kernel that runs many transforms
// with the same thread layout.  NoRegTw: every stage reads the table.
template <int R, int NS_>
struct RegTw {
    static constexpr int kNS = NS_;
    float2 w[R - 1];
};
struct NoRegTw { static constexpr int kNS = 0; };

// Stage compute: registers v[b*R + r] hold input r of butterfly j = t + b*TPT.
// W_16^r = exp(-2 pi i r / 16), r = 0 .. 7.
__device__ __forceinline__ float2 w16(int r) {
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
    switch (r) {
        case 1: return make_float2(c1, -s1);
        case 2: return make_float2(h, -h);
        case 3: return make_float2(s1, -c1);
        case 5: return make_float2(-s1, -c1);
        case 6: return make_float2(-h, -h);
        case 7: return make_float2(-c1, -s1);
        default: return make_float2(1.f, 0.f);
    }
}

// DER: in a radix-8 stage where a thread owns two butterflies whose jm differ
// by TPT = NS / 2, the second butterfly's twiddles are derived from the
// first's, W_{8 NS}^{(jm + NS/2) r} = W_{8 NS}^{jm r} W_16^r (a product with
// a constant: one rounding more, no shared-memory load).
template <int N, int E, int R, int NS, int OFF, bool INV, class RT = NoRegTw, bool DER = false>
__device__ __forceinline__ void stage(float2 (&v)[E], int t, const float2* tw, const RT& rt = RT{}) {
    constexpr int TPT = N / E;
    constexpr bool kReg = NS > 1 && RT::kNS == NS;
    static_assert(!kReg || ((E == R || TPT % NS == 0) && std::is_same<RT, RegTw<R, NS>>::value),
                  "register twiddles: one jm per thread in this stage");
    constexpr bool kDer = DER && !kReg && NS > 1 && R == 8 && E == 2 * R && NS == 2 * TPT;
    float2 w0[R - 1];
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        float2* x = v + b * R;
        if (NS > 1) {
            const int j = t + b * TPT;
            const int jm = j % NS;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w;
                if constexpr (kReg) {
                    w = rt.w[r - 1];
                } else if (kDer && b == 1) {
                    const float2 a = w0[r - 1];
                    w = r == 4 ? make_float2(a.y, -a.x) : cmul(a, w16(r));
                } else {
                    w = tw[OFF + (r - 1) * NS + jm];
                    if (kDer) w0[r - 1] = w;
                }
                if (INV) w.y = -w.y;
                x[r] = cmul(x[r], w);
            }
        }
        Dft<R, INV>::run(x);
    }
}

template <int N, int E, int R, int NS, int X, class L>
__device__ __forceinline__ void write_out(const float2 (&v)[E], float2* buf, int t, L lay) {
    constexpr int TPT = N / E;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        const int j = t + b * TPT;
        const int base = (j / NS) * NS * R + (j % NS);
        if constexpr (IsPadded<L>::value) {
            using F = typename L::template Pad<X>;
            // base + r NS, base = (j / NS) NS R + j mod NS: (base mod kRun) + (r NS mod kRun) < kRun
            // holds when NS is a multiple of kRun; when NS divides kRun and NS R is a multiple of
            // kRun (the offsets reach at most kRun - NS, j mod NS at most NS - 1); and when NS R
            // divides kRun (base + r NS stays inside one block of NS R positions)
            constexpr int K = F::kRun, M = NS * R;
            static_assert(NS % K == 0 || (K % NS == 0 && M % K == 0) || (M <= K && K % M == 0),
                          "padded exchange needs offsets that do not carry");
            const int pb = F::map(base);
#pragma unroll
            for (int r = 0; r < R; ++r) buf[lay.template at<F>(pb, r * NS)] = v[b * R + r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) buf[lay(base + r * NS)] = v[b * R + r];
        }
    }
}

template <int N, int E, int R, int X, class L>
__device__ __forceinline__ void read_in(float2 (&v)[E], const float2* buf, int t, L lay) {
    constexpr int TPT = N / E;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        const int j = t + b * TPT;
        if constexpr (IsPadded<L>::value) {
            using F = typename L::template Pad<X>;
            // j + r N/R with j < N/R: no carry when N/R is a multiple of kRun (offsets 0 mod
            // kRun) or divides kRun (offsets at most kRun - N/R, j at most N/R - 1)
            static_assert((N / R) % F::kRun == 0 || F::kRun % (N / R) == 0,
                          "padded exchange needs offsets that do not carry");
            const int pb = F::map(j);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = buf[lay.template at<F>(pb, r * (N / R))];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = buf[lay(j + r * (N / R))];
        }
    }
}

// canonical (position t + TPT m in v[m]) <-> stage order (b, r) for the first
// / last stage of radix R: position t + TPT (b + r E/R).
template <int E, int R>
__device__ __forceinline__ void canon_to_stage(float2 (&v)[E]) {
    float2 tmp[E];
#pragma unroll
    for (int b = 0; b < E / R; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) tmp[b * R + r] = v[b + r * (E / R)];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = tmp[m];
}
template <int E, int R>
__device__ __forceinline__ void stage_to_canon(float2 (&v)[E]) {
    float2 tmp[E];
#pragma unroll
    for (int b = 0; b < E / R; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) tmp[b + r * (E / R)] = v[b * R + r];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = tmp[m];
}

// Barrier of the threads that share a transform's exchange buffer: the whole
// block, one named barrier (ids 1 .. 15, `count` threads, a multiple of 32)
// per group of transforms whose buffers no other threads touch, or the warp.
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct NamedSync {
    int id, count;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
    }
};
// Transforms whose threads all lie in one warp.
struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

template <int N, int E, bool INV, int NS, int OFF, class L, class S, class RT, bool DER, int X, int R, int... Rest>
__device__ __forceinline__ void run_stages(float2 (&v)[E], float2* b0, float2* b1, int t,
                                           const float2* tw, L lay, S sync, const RT& rt) {
    if constexpr (sizeof...(Rest) > 0) {
        stage<N, E, R, NS, OFF, INV, RT, DER>(v, t, tw, rt);
        constexpr int RN = First<Rest...>::value;
        constexpr int NEXT_OFF = OFF + (NS > 1 ? (R - 1) * NS : 0);
        if (b0 == b1) sync();            // one buffer: the previous exchange's reads come first
        write_out<N, E, R, NS, X>(v, b0, t, lay);
        sync();
        read_in<N, E, RN, X>(v, b0, t, lay);
        run_stages<N, E, INV, NS * R, NEXT_OFF, L, S, RT, DER, X + 1, Rest...>(v, b1, b0, t, tw, lay, sync, rt);
    } else {
        stage<N, E, R, NS, OFF, INV, RT, DER>(v, t, tw, rt);
        stage_to_canon<E, R>(v);
    }
}

template <int N, int E, bool INV, class L, class S, class RT, bool DER, int R0, int... Rs>
__device__ __forceinline__ void transform_impl(Radices<R0, Rs...>, float2 (&v)[E],
                                               float2* b0, float2* b1, int t, const float2* tw,
                                               L lay, S sync, const RT& rt) {
    canon_to_stage<E, R0>(v);
    run_stages<N, E, INV, 1, 0, L, S, RT, DER, 0, R0, Rs...>(v, b0, b1, t, tw, lay, sync, rt);
}

// Plans whose paired butterflies derive their twiddles (see stage).
template <class P, class = void>
struct DerivesTw { static constexpr bool value = false; };
template <class P>
struct DerivesTw<P, decltype(void(P::kDeriveTw))> { static constexpr bool value = P::kDeriveTw; };

// The stage of radices Rs whose twiddles a thread of a plan with TPT threads
// per transform can hold in registers: the last stage when a thread owns one
// butterfly there (E == its radix), else the latest stage with NS > 1 whose NS
// divides TPT (all of a thread's butterflies share jm); ns = 0 if none.
template <int E, int TPT, int NS, int OFF, int R, int... Rest>
struct RegStageOf {
    static constexpr int kNextOff = OFF + (NS > 1 ? (R - 1) * NS : 0);
    static constexpr bool kLast = sizeof...(Rest) == 0;
    static constexpr bool kHere = NS > 1 && ((kLast && E == R) || TPT % NS == 0);
    template <bool LAST, int Dummy = 0>
    struct Later { static constexpr int radix = 0, ns = 0, off = 0; };
    template <int Dummy>
    struct Later<false, Dummy> : RegStageOf<E, TPT, NS * R, kNextOff, Rest...> {};
    using L = Later<kLast>;
    static constexpr bool kLater = L::ns > 0;
    static constexpr int radix = kLater ? L::radix : (kHere ? R : 0);
    static constexpr int ns = kLater ? L::ns : (kHere ? NS : 0);
    static constexpr int off = kLater ? L::off : (kHere ? OFF : 0);
};
// RegStage for a transform of N points by plan P (TPT = N / E threads).
template <class P, int N, class Rs = typename P::R>
struct RegStageN;
template <class P, int N, int... Rs>
struct RegStageN<P, N, Radices<Rs...>> : RegStageOf<P::E, N / P::E, 1, 0, Rs...> {};

// Register twiddles type of plan P at N points (NoRegTw when no stage qualifies).
template <class P, int N>
using RegTwOf = typename std::conditional<(RegStageN<P, N>::ns > 0),
                                          RegTw<(RegStageN<P, N>::radix > 1 ? RegStageN<P, N>::radix : 2),
                                                RegStageN<P, N>::ns>,
                                          NoRegTw>::type;

// Load the register twiddles of plan P (N points) for thread t from its table
// tw (shared memory); an empty NoRegTw when no stage qualifies.
template <class P, int N>
__device__ __forceinline__ RegTwOf<P, N> load_reg_tw(const float2* tw, int t) {
    using RS = RegStageN<P, N>;
    RegTwOf<P, N> rt{};
    if constexpr (RS::ns > 0) {
        const int jm = t % RS::ns;
#pragma unroll
        for (int r = 1; r < RS::radix; ++r) rt.w[r - 1] = tw[RS::off + (r - 1) * RS::ns + jm];
    }
    return rt;
}

// Size of the per-stage twiddle table of a plan.
template <int NS, int R, int... Rest>
constexpr int tw_entries() {
    constexpr int here = NS > 1 ? (R - 1) * NS : 0;
    if constexpr (sizeof...(Rest) > 0) return here + tw_entries<NS * R, Rest...>();
    else return here;
}
template <int... Rs>
constexpr int tw_entries_of(Radices<Rs...>) { return tw_entries<1, Rs...>(); }
template <int N>
struct TwSize { static constexpr int value = tw_entries_of(typename Plan<N>::R{}); };

// Fill the per-stage twiddle table of Plan<N> in FP64 (threads tid of nthr).
template <int NS, int OFF, int R, int... Rest>
__device__ void fill_twiddles_impl(float2* tw, int tid, int nthr) {
    if constexpr (NS > 1) {
        for (int e = tid; e < (R - 1) * NS; e += nthr) {
            const int r = 1 + e / NS, jm = e % NS;
            double sn, cs;
            sincospi(-2.0 * (double)(jm * r) / (double)(NS * R), &sn, &cs);
            tw[OFF + e] = make_float2((float)cs, (float)sn);
        }
    }
    if constexpr (sizeof...(Rest) > 0)
        fill_twiddles_impl<NS * R, OFF + (NS > 1 ? (R - 1) * NS : 0), Rest...>(tw, tid, nthr);
}
template <int... Rs>
__device__ void fill_twiddles_of(Radices<Rs...>, float2* tw, int tid, int nthr) {
    fill_twiddles_impl<1, 0, Rs...>(tw, tid, nthr);
}
template <int N>
__device__ void fill_twiddles(float2* tw, int tid, int nthr) {
    fill_twiddles_of(typename Plan<N>::R{}, tw, tid, nthr);
}

// Full length-N transform of the values held in canonical order by the TPT
// threads of one transform.  Every thread of the block must call it the same
// number of times (it contains barriers: __syncthreads, or the named barrier
// `sync` of the threads sharing the buffers).  tw: the plan's per-stage
// twiddle table (TwSize<N> entries), normally staged in shared memory.
// With two buffers a leading barrier separates the last shared-memory reads
// of a previous transform from the first writes of this one (plans with one
// exchange would otherwise reuse a buffer without a barrier in between).  With
// one buffer (b0 == b1) every exchange already starts with a barrier before
// its writes, and the first stage touches no shared memory but the twiddles
// (read-only), so no leading barrier is needed.
template <int N, bool INV, class L, class S = BlockSync>
__device__ __forceinline__ void transform(float2 (&v)[Plan<N>::E], float2* b0, float2* b1, int t,
                                          const float2* tw, L lay, S sync = S{}) {
    if (b0 != b1) sync();
    transform_impl<N, Plan<N>::E, INV, L, S, NoRegTw, false>(typename Plan<N>::R{}, v, b0, b1, t, tw, lay, sync,
                                                             NoRegTw{});
}

// The same with an explicit plan P (P::E values per thread, radices P::R; its
// twiddle table is that of Plan<N> when the radices agree).
// rt: NoRegTw, or one stage's twiddles from load_reg_tw<P, N>.
template <class P, int N, bool INV, class L, class S, class RT = NoRegTw>
__device__ __forceinline__ void transform_plan(float2 (&v)[P::E], float2* b0, float2* b1, int t,
                                               const float2* tw, L lay, S sync, const RT& rt = RT{}) {
    if (b0 != b1) sync();
    transform_impl<N, P::E, INV, L, S, RT, DerivesTw<P>::value>(typename P::R{}, v, b0, b1, t, tw, lay, sync, rt);
}

}  // namespace fft
}  // namespace tacaw
