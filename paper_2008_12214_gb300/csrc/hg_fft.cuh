// hg_fft.cuh -- register/shared-memory mixed-radix (2/3/5) Stockham line FFT
// for sm_103a, the engine under every pass of the hologram iteration.
//
// The transform is the unnormalised 1D DFT X[k] = sum_n x[n] W_N^{nk},
// W_N = exp(DIR 2 pi i / N) (DIR = -1 forward, +1 inverse); the unitary
// 1/sqrt(Nx Ny) of the paper's eqs. (fouriertrans2d5c/d) (Section 2) is applied
// by the callers where a value is consumed.
//
// Decomposition.  N = R_0 R_1 ... R_{m-1}.  Before stage s the data is
// P_s = R_0...R_{s-1} independent sub-transforms of length N / P_s stored
// Stockham (autosort) style: sub-transform kappa, element nu at address
// kappa + P_s nu.  Stage s writes nu = nu1 + Q_s nu2 (Q_s = N / (P_s R_s)),
// takes the R_s-point DFT over nu2 for every (kappa, nu1), multiplies output
// k by W_N^{P_s nu1 k} and stores it at kappa + P_s k + P_s R_s nu1.  After the
// last stage the addresses are the natural output order.  Butterfly
// b = kappa + P_s nu1 reads addresses b + (N / R_s) j, so consecutive threads
// read consecutive addresses at every stage.
//
// Threads.  TL threads serve one line and each holds E = N / TL samples,
// thread t holding samples t + TL e (e < E) at entry and at exit of the line
// transform (stage 0 reads its butterflies straight from those registers; the
// last stage writes back into them when R_last divides E, otherwise through
// shared memory).  Middle stages exchange through shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace hg {

// ----------------------------------------------------------------- helpers

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * w
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// a * conj(w)
__device__ __forceinline__ float2 cmulc(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}
// a * (DIR i)
template <int DIR>
__device__ __forceinline__ float2 mul_di(float2 a) {
    return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// a * w^{-DIR}... : multiply by the stage root, given the table value of the
// forward root exp(-2 pi i e / N): forward keeps it, inverse conjugates.
template <int DIR>
__device__ __forceinline__ float2 cmul_root(float2 a, float2 wfwd) {
    return DIR < 0 ? cmul(a, wfwd) : cmulc(a, wfwd);
}

// ------------------------------------------------ compile-time unit roots
// cos / sin of 2 pi e / R evaluated at compile time: the angle is split by
// exact integer arithmetic into an octant q (multiples of pi/4) and a residual
// x in [0, pi/4), the residual's sine and cosine come from their Taylor series
// (terms to x^25, far below double rounding for |x| <= pi/4), and the octant
// is restored with the angle-addition identities.

constexpr double kPiOver4 = 0.78539816339744830961566084581987572;

__host__ __device__ constexpr double taylor_sin(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int k = 1; k <= 12; ++k) {
        term *= -x2 / double((2 * k) * (2 * k + 1));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k <= 12; ++k) {
        term *= -x2 / double((2 * k - 1) * (2 * k));
        sum += term;
    }
    return sum;
}

struct dpair {
    double c, s;
};

// (cos, sin)(2 pi e / R)
__host__ __device__ constexpr dpair unit_root(long e, long R) {
    e %= R;
    if (e < 0) e += R;
    const long q = (8 * e) / R;      // octant, 0..7
    const long rem = 8 * e - q * R;  // angle = pi/4 (q + rem/R)
    const double x = kPiOver4 * double(rem) / double(R);
    const double y = kPiOver4 * double(R - rem) / double(R);  // pi/4 - x
    const double cx = taylor_cos(x), sx = taylor_sin(x), cy = taylor_cos(y), sy = taylor_sin(y);
    switch (q) {
        case 0: return {cx, sx};
        case 1: return {sy, cy};
        case 2: return {-sx, cx};
        case 3: return {-cy, sy};
        case 4: return {-cx, -sx};
        case 5: return {-sy, -cy};
        case 6: return {sx, -cx};
        default: return {cy, -sy};
    }
}

// v * W_R^E with W_R = exp(DIR 2 pi i / R), E a compile-time exponent.
template <int R, int E, int DIR>
__device__ __forceinline__ float2 twc(float2 v) {
    constexpr int e = ((E % R) + R) % R;
    if constexpr (e == 0) {
        return v;
    } else if constexpr (4 * e == R) {
        return mul_di<DIR>(v);
    } else if constexpr (2 * e == R) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (4 * e == 3 * R) {
        return mul_di<-DIR>(v);
    } else {
        constexpr dpair w = unit_root(e, R);
        constexpr float c = float(w.c);
        constexpr float s = float(DIR > 0 ? w.s : -w.s);
        return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
    }
}

// --------------------------------------------------- in-register DFT codelets

template <int R>
__host__ __device__ constexpr int first_factor() {
    if constexpr (R % 4 == 0 && R != 4) return 4;
    else if constexpr (R % 2 == 0) return 2;
    else if constexpr (R % 3 == 0) return 3;
    else return 5;
}

// In-place R-point DFT of x[0..R) held in registers (all indices compile-time).
template <int R, int DIR>
__device__ __forceinline__ void dft(float2 *x) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        const float2 a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    } else if constexpr (R == 3) {
        // W3 = -1/2 + DIR i sqrt(3)/2
        const float2 t1 = cadd(x[1], x[2]);
        const float2 t2 = make_float2(fmaf(-0.5f, t1.x, x[0].x), fmaf(-0.5f, t1.y, x[0].y));
        const float2 t3 = mul_di<DIR>(cscale(csub(x[1], x[2]), 0.86602540378443864676f));
        x[0] = cadd(x[0], t1);
        x[1] = cadd(t2, t3);
        x[2] = csub(t2, t3);
    } else if constexpr (R == 4) {
        const float2 a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
        const float2 c = cadd(x[1], x[3]), d = mul_di<DIR>(csub(x[1], x[3]));
        x[0] = cadd(a, c);
        x[2] = csub(a, c);
        x[1] = cadd(b, d);
        x[3] = csub(b, d);
    } else if constexpr (R == 5) {
        // cos / sin of 2 pi/5 and 4 pi/5
        constexpr float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
        constexpr float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
        const float2 a1 = cadd(x[1], x[4]), a2 = cadd(x[2], x[3]);
        const float2 b1 = csub(x[1], x[4]), b2 = csub(x[2], x[3]);
        const float2 x0 = x[0];
        const float2 p1 = make_float2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
        const float2 p2 = make_float2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
        const float2 q1 = mul_di<DIR>(make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
        const float2 q2 = mul_di<DIR>(make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
        x[0] = cadd(x0, cadd(a1, a2));
        x[1] = cadd(p1, q1);
        x[4] = csub(p1, q1);
        x[2] = cadd(p2, q2);
        x[3] = csub(p2, q2);
    } else {
        // R = A B, n = n1 + B n2, k = k2 + A k1 (four-step in registers)
        constexpr int A = first_factor<R>();
        constexpr int B = R / A;
        float2 y[R];  // y[k2 * B + n1]
        static_for<0, B>([&](auto n1c) {
            constexpr int n1 = decltype(n1c)::value;
            float2 t[A];
            static_for<0, A>([&](auto n2c) {
                constexpr int n2 = decltype(n2c)::value;
                t[n2] = x[n1 + B * n2];
            });
            dft<A, DIR>(t);
            static_for<0, A>([&](auto k2c) {
                constexpr int k2 = decltype(k2c)::value;
                y[k2 * B + n1] = twc<R, n1 * k2, DIR>(t[k2]);
            });
        });
        static_for<0, A>([&](auto k2c) {
            constexpr int k2 = decltype(k2c)::value;
            dft<B, DIR>(y + k2 * B);
            static_for<0, B>([&](auto k1c) {
                constexpr int k1 = decltype(k1c)::value;
                x[k2 + A * k1] = y[k2 * B + k1];
            });
        });
    }
}

// ------------------------------------------------------------ line plans

template <int N_, int TL_, int PAD_, int... Rs>
struct Plan {
    static constexpr int N = N_;
    static constexpr int TL = TL_;
    static constexpr int E = N_ / TL_;
    static constexpr int PAD = PAD_;
    static constexpr int NS = sizeof...(Rs);
    static constexpr int R[NS] = {Rs...};
    static constexpr int SLOTS = N_ + N_ / PAD_;  // padded complex slots per line
    __host__ __device__ static constexpr int prodR(int s) {
        int p = 1;
        for (int i = 0; i < s; ++i) p *= R[i];
        return p;
    }
    static constexpr bool LAST_TO_REGS =
        (E % R[NS - 1] == 0) && ((N_ / R[NS - 1]) % TL_ == 0);
    static_assert(prodR(NS) == N_, "radices must multiply to N");
    static_assert(N_ % TL_ == 0, "threads per line must divide N");
    static_assert(E % R[0] == 0, "first radix must divide the samples per thread");
};

// Shared-memory layouts of one line during the exchanges (consecutive
// addresses STRIDE float2 apart).
//  Pad:      one pad slot every P::PAD addresses (needs P::SLOTS slots per
//            line); breaks the stride-R bank pattern of stage 0's stores.
//  Swz<L>:   a ^ ((a >> L) & (2^L - 1)): a permutation inside every aligned
//            block of 2^L addresses (needs N slots, N a multiple of 2^L), so a
//            line can be exchanged in place in the buffer it was loaded into.
struct Pad {
    template <class P>
    __device__ __forceinline__ static int idx(int a) { return a + a / P::PAD; }
};
template <int L>
struct Swz {
    template <class P>
    __device__ __forceinline__ static int idx(int a) {
        static_assert(P::N % (1 << L) == 0, "swizzle blocks must tile the line");
        return a ^ ((a >> L) & ((1 << L) - 1));
    }
};

template <class P, int STRIDE, class LAY = Pad>
__device__ __forceinline__ float2 &slot(float2 *base, int a) {
    return base[LAY::template idx<P>(a) * STRIDE];
}

// Stage 0: butterflies straight from the registers v; the result goes to
// shared memory (or back to v when the plan has one stage).
template <class P, int DIR, int STRIDE, class LAY>
__device__ __forceinline__ void stage_first(float2 (&v)[P::E], float2 *smb,
                                            const float2 *__restrict__ tw, int t) {
    constexpr int R = P::R[0];
    constexpr int NB = P::E / R;
    static_for<0, NB>([&](auto uc) {
        constexpr int u = decltype(uc)::value;
        float2 x[R];
        static_for<0, R>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            x[j] = v[u + NB * j];
        });
        dft<R, DIR>(x);
        if constexpr (P::NS == 1) {
            static_for<0, R>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                v[u + NB * k] = x[k];
            });
        } else {
            const int b = t + P::TL * u;  // nu1 (P_0 = 1, kappa = 0)
            static_for<1, R>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                x[k] = cmul_root<DIR>(x[k], __ldg(tw + b * k));
            });
            static_for<0, R>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                slot<P, STRIDE, LAY>(smb, k + R * b) = x[k];
            });
        }
    });
}

// Stage S >= 1: read from shared memory, transform, then write to shared
// memory or (last stage with TO_REGS) into v.
template <class P, int S, int DIR, int STRIDE, bool TO_REGS, class LAY, class SYNC>
__device__ __forceinline__ void stage_next(float2 (&v)[P::E], float2 *smb,
                                           const float2 *__restrict__ tw, int t, SYNC sync) {
    constexpr int R = P::R[S];
    constexpr int M = P::N / R;        // butterflies per line
    constexpr int PS = P::prodR(S);    // P_s
    constexpr int NB = (M + P::TL - 1) / P::TL;
    constexpr bool EXACT = (M % P::TL) == 0;
    float2 x[NB][R];
    static_for<0, NB>([&](auto uc) {
        constexpr int u = decltype(uc)::value;
        const int b = t + P::TL * u;
        if (EXACT || b < M) {
            static_for<0, R>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                x[u][j] = slot<P, STRIDE, LAY>(smb, b + M * j);
            });
        }
    });
    if constexpr (!TO_REGS) sync();
    static_for<0, NB>([&](auto uc) {
        constexpr int u = decltype(uc)::value;
        const int b = t + P::TL * u;
        if (EXACT || b < M) {
            dft<R, DIR>(x[u]);
            if constexpr (TO_REGS) {
                static_for<0, R>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    v[u + NB * k] = x[u][k];
                });
            } else {
                const int kap = b % PS, nu1 = b / PS;
                if constexpr (S < P::NS - 1) {
                    static_for<1, R>([&](auto kc) {
                        constexpr int k = decltype(kc)::value;
                        x[u][k] = cmul_root<DIR>(x[u][k], __ldg(tw + PS * nu1 * k));
                    });
                }
                static_for<0, R>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    slot<P, STRIDE, LAY>(smb, kap + PS * k + PS * R * nu1) = x[u][k];
                });
            }
        }
    });
    if constexpr (!TO_REGS) sync();
}

// A plan whose stage roots are loaded afresh by every line transform.  In a
// persistent kernel each thread's roots are the same for every line it
// transforms, so the compiler keeps them in registers across the whole loop
// (about 2 (R_0 - 1) + 2 (R_1 - 1) registers for a three-stage plan); this
// wrapper trades those registers for L1-resident reloads, raising the number
// of warps an SM can hold.
template <class P>
struct Reload : P {
    static constexpr bool TW_RELOAD = true;
};
template <class P, class = void>
struct tw_reload : std::false_type {};
template <class P>
struct tw_reload<P, std::void_t<decltype(P::TW_RELOAD)>> : std::bool_constant<P::TW_RELOAD> {};

// Whole line transform: thread t holds samples t + TL e in v on entry and the
// transform's outputs t + TL e on exit.  `sync` must order shared-memory
// accesses of all threads of the line.  Shared memory may be reused between
// calls without further synchronisation.
template <class P, int DIR, int STRIDE, class LAY = Pad, class SYNC>
__device__ __forceinline__ void line_fft(float2 (&v)[P::E], float2 *smb,
                                         const float2 *__restrict__ tw, int t, SYNC sync) {
    if constexpr (tw_reload<P>::value) {
        // an opaque copy of the table pointer: loads through it cannot be
        // hoisted out of the caller's loop
        asm volatile("mov.b64 %0, %0;" : "+l"(tw));
    }
    if constexpr (P::NS == 1) {
        stage_first<P, DIR, STRIDE, LAY>(v, smb, tw, t);
    } else {
        sync();  // earlier readers of this line's shared memory are done
        stage_first<P, DIR, STRIDE, LAY>(v, smb, tw, t);
        sync();
        static_for<1, P::NS>([&](auto sc) {
            constexpr int S = decltype(sc)::value;
            constexpr bool to_regs = (S == P::NS - 1) && P::LAST_TO_REGS;
            stage_next<P, S, DIR, STRIDE, to_regs, LAY>(v, smb, tw, t, sync);
        });
        if constexpr (!P::LAST_TO_REGS) {
            static_for<0, P::E>([&](auto ec) {
                constexpr int e = decltype(ec)::value;
                v[e] = slot<P, STRIDE, LAY>(smb, t + P::TL * e);
            });
        }
    }
}

// ------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten rounds
// of two 32x32->64 multiplications by the Philox constants with the high
// halves mixed into the other words and the key, the key advanced by the Weyl
// constants between rounds.  Returns output word 0.
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return c0;
}

// All four output words of the same generator.
__device__ __forceinline__ uint4 philox4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                         uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// The random phase of replay pixel r (= y nx + x) of a drawn phase map, as
// 2u with u = (word >> 8) 2^-24 in [0, 1), ready for sincospif: every group
// of four consecutive pixels shares one generator call, counter {r / 4, sub,
// target, stream}, pixel r taking output word r mod 4.
__device__ __forceinline__ float philox_phase2u(uint32_t r, uint32_t sub, uint32_t target, uint32_t stream,
                                                uint32_t k0, uint32_t k1) {
    const uint4 w = philox4(r >> 2, sub, target, stream, k0, k1);
    const uint32_t q = r & 3u;
    const uint32_t v = q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w;
    return (float)(v >> 8) * (1.0f / 8388608.0f);
}

// Output words 0 and 1 of the same generator.
__device__ __forceinline__ uint2 philox_words01(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint2(c0, c1);
}

}  // namespace hg
