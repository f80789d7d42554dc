// Register-group engine shared by the blocking-section kernels: gates applied to 2^R amplitudes
// held in registers, with the amplitudes read from / written to a chunk in shared memory
// (swizzled layout, host-chosen lane layouts; see sv_internal.h for the swizzle table).
#pragma once
#include <stdint.h>

#include "ptx.cuh"
#include "sv_internal.h"

namespace sv {
namespace {

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

// Swizzle patterns V[k] (see sv_internal.h); the host picks lane layouts from the same table.
__constant__ int c_swz64[24] = {SV_SWZ64_LIST};
__constant__ int c_swz128[24] = {SV_SWZ128_LIST};

// Lowest set bit of a non-zero loop index that unrolling makes a constant.  Indexing a step table
// with __ffs(b) - 1 is not folded and puts the table in local memory; this expression is.
__host__ __device__ constexpr int low_bit(int b) {
    return (b & 1) ? 0 : (b & 2) ? 1 : (b & 4) ? 2 : (b & 8) ? 3 : 4;
}

__device__ __forceinline__ int insert0(int x, int p) { return ((x >> p) << (p + 1)) | (x & ((1 << p) - 1)); }

template <typename T>
__device__ __forceinline__ void cmul_acc(T &yr, T &yi, T mr, T mi, T xr, T xi) {
    yr = fma(mr, xr, yr);
    yr = fma(-mi, xi, yr);
    yi = fma(mr, xi, yi);
    yi = fma(mi, xr, yi);
}

// ---- explicit shared-memory access with 32-bit shared addresses.  Chunk data goes through
// volatile accesses (ordered with the barriers); the section program is read-only after the
// kernel's first barrier, so its loads are pure and the compiler may reuse them across groups.
template <typename T> struct SM;
template <> struct SM<float> {
    static __device__ __forceinline__ void ld(uint32_t a, float &x, float &y) {
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a));
    }
    static __device__ __forceinline__ void st(uint32_t a, float x, float y) {
        asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x), "f"(y) : "memory");
    }
    static __device__ __forceinline__ void ldc4(uint32_t a, float &x, float &y, float &z, float &w) {
        asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x), "=f"(y), "=f"(z), "=f"(w) : "r"(a));
    }
};
template <> struct SM<double> {
    static __device__ __forceinline__ void ld(uint32_t a, double &x, double &y) {
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(x), "=d"(y) : "r"(a));
    }
    static __device__ __forceinline__ void st(uint32_t a, double x, double y) {
        asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(x), "d"(y) : "memory");
    }
    static __device__ __forceinline__ void ldc4(uint32_t a, double &x, double &y, double &z, double &w) {
        asm("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(x), "=d"(y) : "r"(a));
        asm("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(z), "=d"(w) : "r"(a + 16));
    }
};

__device__ __forceinline__ int lds_s8(uint32_t a) {
    int v;
    asm volatile("ld.shared.s8 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ int lds_s16(uint32_t a) {
    int v;
    asm volatile("ld.shared.s16 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ int lds_s32(uint32_t a) {
    int v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void ldc_i4(uint32_t a, int &x, int &y, int &z, int &w) {
    asm("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(x), "=r"(y), "=r"(z), "=r"(w) : "r"(a));
}

template <typename T, int K>
__device__ __forceinline__ void load_mat(uint32_t a, T (&m)[K]) {
#pragma unroll
    for (int k = 0; k < K; k += 4) SM<T>::ldc4(a + k * (uint32_t)sizeof(T), m[k], m[k + 1], m[k + 2], m[k + 3]);
}

template <typename T, int NA, int A>
__device__ __forceinline__ void ap_dense1(T (&r)[NA], T (&i)[NA], uint32_t ma) {
    T m[8];
    load_mat<T, 8>(ma, m);
#pragma unroll
    for (int x = 0; x < NA; ++x) {
        if (x & (1 << A)) continue;
        const int y = x | (1 << A);
        const T ar = r[x], ai = i[x], br = r[y], bi = i[y];
        T pr = 0, pi = 0, qr = 0, qi = 0;
        cmul_acc(pr, pi, m[0], m[1], ar, ai);
        cmul_acc(pr, pi, m[2], m[3], br, bi);
        cmul_acc(qr, qi, m[4], m[5], ar, ai);
        cmul_acc(qr, qi, m[6], m[7], br, bi);
        r[x] = pr; i[x] = pi; r[y] = qr; i[y] = qi;
    }
}

// Diagonal gates.  Complex128 sections are FP64-bound on this GPU, so there an entry of exactly
// 1 leaves its amplitudes alone (a controlled phase touches a quarter of them; the test is
// uniform over the warp); complex64 multiplies through, the branch-free form being faster.
template <typename T>
__device__ __forceinline__ void scale_amp(T &re, T &im, T dr, T di) {
    const T xr = re, xi = im;
    re = fma(dr, xr, -di * xi);
    im = fma(dr, xi, di * xr);
}

template <typename T, int NA, int A>
__device__ __forceinline__ void ap_diag1(T (&r)[NA], T (&i)[NA], uint32_t ma) {
    T d[4];
    load_mat<T, 4>(ma, d);
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const T dr = d[2 * l], di = d[2 * l + 1];
            if (di == T(0) && dr == T(1)) continue;
#pragma unroll
            for (int x = 0; x < NA; ++x)
                if (((x >> A) & 1) == l) scale_amp(r[x], i[x], dr, di);
        }
    } else {
#pragma unroll
        for (int x = 0; x < NA; ++x) {
            const int l = (x >> A) & 1;
            scale_amp(r[x], i[x], d[2 * l], d[2 * l + 1]);
        }
    }
}

template <typename T, int NA, int A, int B>
__device__ __forceinline__ void ap_dense2(T (&r)[NA], T (&i)[NA], uint32_t ma) {
    T mm[32];
    load_mat<T, 32>(ma, mm);
#pragma unroll
    for (int x = 0; x < NA; ++x) {
        if (x & ((1 << A) | (1 << B))) continue;
        const int id[4] = {x, x | (1 << A), x | (1 << B), x | (1 << A) | (1 << B)};
        T xr[4], xi[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { xr[k] = r[id[k]]; xi[k] = i[id[k]]; }
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            T yr = 0, yi = 0;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) cmul_acc(yr, yi, mm[2 * (4 * rr + cc)], mm[2 * (4 * rr + cc) + 1], xr[cc], xi[cc]);
            r[id[rr]] = yr;
            i[id[rr]] = yi;
        }
    }
}

template <typename T, int NA, int A, int B>
__device__ __forceinline__ void ap_diag2(T (&r)[NA], T (&i)[NA], uint32_t ma) {
    T d[8];
    load_mat<T, 8>(ma, d);
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const T dr = d[2 * l], di = d[2 * l + 1];
            if (di == T(0) && dr == T(1)) continue;
#pragma unroll
            for (int x = 0; x < NA; ++x)
                if ((((x >> A) & 1) | (((x >> B) & 1) << 1)) == l) scale_amp(r[x], i[x], dr, di);
        }
    } else {
#pragma unroll
        for (int x = 0; x < NA; ++x) {
            const int l = ((x >> A) & 1) | (((x >> B) & 1) << 1);
            scale_amp(r[x], i[x], d[2 * l], d[2 * l + 1]);
        }
    }
}

template <typename T, int NA, int A, int B>
__device__ __forceinline__ void ap_perm2(T (&r)[NA], T (&i)[NA], uint32_t ma) {
    T pm[4];
    load_mat<T, 4>(ma, pm);
    const int p0 = (int)pm[0], p1 = (int)pm[1], p2 = (int)pm[2], p3 = (int)pm[3];
#pragma unroll
    for (int x = 0; x < NA; ++x) {
        if (x & ((1 << A) | (1 << B))) continue;
        const int id[4] = {x, x | (1 << A), x | (1 << B), x | (1 << A) | (1 << B)};
        T xr[4], xi[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { xr[k] = r[id[k]]; xi[k] = i[id[k]]; }
        const int p[4] = {p0, p1, p2, p3};
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int s = p[rr];
            r[id[rr]] = s == 0 ? xr[0] : s == 1 ? xr[1] : s == 2 ? xr[2] : xr[3];
            i[id[rr]] = s == 0 ? xi[0] : s == 1 ? xi[1] : s == 2 ? xi[2] : xi[3];
        }
    }
}

// Bit flip on register bit A: a pure exchange of registers (no arithmetic).
template <typename T, int NA, int A>
__device__ __forceinline__ void ap_x1(T (&r)[NA], T (&i)[NA]) {
#pragma unroll
    for (int x = 0; x < NA; ++x) {
        if (x & (1 << A)) continue;
        const int y = x | (1 << A);
        T t = r[x]; r[x] = r[y]; r[y] = t;
        t = i[x]; i[x] = i[y]; i[y] = t;
    }
}

// Exchange of the local two-qubit basis states U and V (index = bit A + 2 * bit B) in every
// 4-amplitude block: CNOT and SWAP, again without arithmetic.
template <typename T, int NA, int A, int B, int U, int V>
__device__ __forceinline__ void ap_xchg2(T (&r)[NA], T (&i)[NA]) {
#pragma unroll
    for (int x = 0; x < NA; ++x) {
        if (x & ((1 << A) | (1 << B))) continue;
        const int id[4] = {x, x | (1 << A), x | (1 << B), x | (1 << A) | (1 << B)};
        T t = r[id[U]]; r[id[U]] = r[id[V]]; r[id[V]] = t;
        t = i[id[U]]; i[id[U]] = i[id[V]]; i[id[V]] = t;
    }
}

// Dispatch a gate on the register bits (a, b) -- compile-time bit positions via templates.
template <typename T, int R, int A>
__device__ __forceinline__ void one(int op, T (&r)[1 << R], T (&i)[1 << R], uint32_t m) {
    if (op == OP_DENSE1) ap_dense1<T, 1 << R, A>(r, i, m);
    else if (op == OP_X1) ap_x1<T, 1 << R, A>(r, i);
    else ap_diag1<T, 1 << R, A>(r, i, m);
}

template <typename T, int R, int A, int B>
__device__ __forceinline__ void two(int op, T (&r)[1 << R], T (&i)[1 << R], uint32_t m) {
    if (op == OP_DENSE2) ap_dense2<T, 1 << R, A, B>(r, i, m);
    else if (op == OP_DIAG2) ap_diag2<T, 1 << R, A, B>(r, i, m);
    else if (op == OP_CXA) ap_xchg2<T, 1 << R, A, B, 1, 3>(r, i);
    else if (op == OP_CXB) ap_xchg2<T, 1 << R, A, B, 2, 3>(r, i);
    else if (op == OP_SWAP2) ap_xchg2<T, 1 << R, A, B, 1, 2>(r, i);
    else ap_perm2<T, 1 << R, A, B>(r, i, m);
}

template <typename T, int R>
__device__ __forceinline__ void apply_gate(int op, int code, uint32_t m, T (&r)[1 << R], T (&i)[1 << R]) {
    if (op == OP_DENSE1 || op == OP_DIAG1 || op == OP_X1) {
        switch (code) {
            case 0: one<T, R, 0>(op, r, i, m); break;
            case 1: one<T, R, 1>(op, r, i, m); break;
            case 2: one<T, R, 2>(op, r, i, m); break;
            case 3: one<T, R, 3>(op, r, i, m); break;
            case 4: if constexpr (R > 4) one<T, R, 4>(op, r, i, m); break;
            default: break;
        }
    } else {
        switch (code) {
            case 0 * 8 + 1: two<T, R, 0, 1>(op, r, i, m); break;
            case 0 * 8 + 2: two<T, R, 0, 2>(op, r, i, m); break;
            case 0 * 8 + 3: two<T, R, 0, 3>(op, r, i, m); break;
            case 1 * 8 + 2: two<T, R, 1, 2>(op, r, i, m); break;
            case 1 * 8 + 3: two<T, R, 1, 3>(op, r, i, m); break;
            case 2 * 8 + 3: two<T, R, 2, 3>(op, r, i, m); break;
            case 0 * 8 + 4: if constexpr (R > 4) two<T, R, 0, 4>(op, r, i, m); break;
            case 1 * 8 + 4: if constexpr (R > 4) two<T, R, 1, 4>(op, r, i, m); break;
            case 2 * 8 + 4: if constexpr (R > 4) two<T, R, 2, 4>(op, r, i, m); break;
            case 3 * 8 + 4: if constexpr (R > 4) two<T, R, 3, 4>(op, r, i, m); break;
            default: break;
        }
    }
}

constexpr int kMaxRest = 8;  // chunk bits above the lanes per register group (c <= R + 5 + 8)

// One register group over the chunk in shared memory.  `buf`, `seg` and `gates` are shared
// addresses of the chunk buffer, the group descriptor and the section's gate records.  Each
// thread handles KU groups at a time so that every gate matrix is read once for all of them.
template <typename T, int R, int NC, int KU>
__device__ __forceinline__ void run_segment(uint32_t buf, uint32_t seg, uint32_t gates, int ctid, const int *swz,
                                            int c, int64_t origin) {
    constexpr int NA = 1 << R;
    constexpr int SH = sizeof(T) == 4 ? 3 : 4;  // log2 bytes per amplitude
    // descriptor (DevSeg layout: pos[8] lane[5] nrest flags r rest[16] g0 g1)
    int po[R], pf[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int p = lds_s8(seg + j);
        po[j] = 1 << p;
        pf[j] = po[j] ^ swz[p];
    }
    const int lane = ctid & 31;
    int lbase = 0, lfb = 0;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int p = lds_s8(seg + 8 + j);
        if ((lane >> j) & 1) { lbase |= 1 << p; lfb ^= swz[p]; }
    }
    const int nrest = lds_s8(seg + 13), flags = lds_s8(seg + 14);
    int rpo[kMaxRest], rpf[kMaxRest];
#pragma unroll
    for (int j = 0; j < kMaxRest; ++j) {
        const int p = j < nrest ? lds_s8(seg + 16 + j) : 0;
        rpo[j] = j < nrest ? 1 << p : 0;
        rpf[j] = j < nrest ? swz[p] : 0;
    }
    const int g0 = lds_s16(seg + 32), g1 = lds_s16(seg + 34);
    const int G = 1 << (c - R);

    // byte steps between a group's amplitudes in Gray-code order: both the natural and the
    // swizzled address are linear over GF(2) in the group index, so each next amplitude is one
    // XOR away (load side and store side may use different layouts)
    uint32_t ld_step[R], st_step[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        ld_step[j] = (uint32_t)((flags & 1) ? po[j] : pf[j]) << SH;
        st_step[j] = (uint32_t)((flags & 2) ? po[j] : pf[j]) << SH;
    }

    for (int gb = ctid; gb < G; gb += NC * KU) {
        T re[KU][NA], im[KU][NA];
        int base[KU], sbase[KU];
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            const int hi = (gb + u * NC) >> 5;
            int bs = lbase, fb = lfb;
#pragma unroll
            for (int j = 0; j < kMaxRest; ++j)
                if ((hi >> j) & 1) { bs |= rpo[j]; fb ^= rpf[j]; }
            base[u] = bs;
            sbase[u] = bs ^ fb;
            if (gb + u * NC < G) {
                // the offset stays below the chunk size, so it is walked by XOR and the buffer
                // base (not aligned to the chunk size) added after
                uint32_t off = (uint32_t)((flags & 1) ? base[u] : sbase[u]) << SH;
#pragma unroll
                for (int b = 0; b < NA; ++b) {
                    if (b) off ^= ld_step[__ffs(b) - 1];
                    const int gidx = b ^ (b >> 1);
                    SM<T>::ld(buf + off, re[u][gidx], im[u][gidx]);
                }
            }
        }
        for (int gi = g0; gi < g1; ++gi) {
            const uint32_t ga = gates + (uint32_t)gi * (uint32_t)sizeof(DevGate<T>);
            int op, ra, rb, code;
            ldc_i4(ga, op, ra, rb, code);
            uint32_t ma = ga + 16;
            if (op == OP_DIAGX) {
                // qubits outside the chunk are fixed over it: read them off the chunk's origin
                const int e0 = rb & 0xFF, e1 = (rb >> 8) & 0xFF;
                int v = (int)((origin >> e0) & 1);
                if (e1 != 0xFF) v |= (int)((origin >> e1) & 1) << 1;
                ma += (uint32_t)(v * 4 * (int)sizeof(T));
                op = OP_DIAG1;  // a phase is encoded as equal entries on register bit 0
            }
#pragma unroll
            for (int u = 0; u < KU; ++u) apply_gate<T, R>(op, code, ma, re[u], im[u]);
        }
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            if (gb + u * NC < G) {
                uint32_t off = (uint32_t)((flags & 2) ? base[u] : sbase[u]) << SH;
#pragma unroll
                for (int b = 0; b < NA; ++b) {
                    if (b) off ^= st_step[__ffs(b) - 1];
                    const int gidx = b ^ (b >> 1);
                    SM<T>::st(buf + off, re[u][gidx], im[u][gidx]);
                }
            }
        }
    }
}


// x rounded to the nearest TF32 value (ties away from zero), as a bit pattern: adding half a TF32
// unit in the last place to the magnitude bits and clearing the 13 dropped bits (a carry into the
// exponent is the correct result).  Two integer operations instead of a conversion instruction.
__device__ __forceinline__ uint32_t tf32_round(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

// Shapes of a tensor-core register group of R bits (complex64): a row is the group's 2^R
// amplitudes as K = 2^(R+1) reals; a tile is 128 rows.  TMEM columns of one tile buffer:
// A_hi [0, K), A_lo [K, 2K), D [2K, 4K).  The B operand (TcGeom::B_BYTES, see TC_B_BYTES) is
// B_hi then B_lo, K-major without swizzle, SBO bytes between 8-column groups, so the two stack
// along N: one descriptor reads [B_hi | B_lo] as a K x 2K matrix.
template <int R>
struct TcGeom {
    static constexpr int NA = 1 << R;
    static constexpr int K = 2 * NA;
    static constexpr int COLS = 4 * K;
    static constexpr int KSTEPS = K / 8;
    static constexpr int SBO = 32 * K;
    static constexpr int B_BYTES = 8 * K * K;
};

template <int NR>
__device__ __forceinline__ void tmem_st_n(uint32_t taddr, const uint32_t *r) {
    if constexpr (NR == 16) {
        ptx::tmem_st16(taddr, r);
    } else {
        ptx::tmem_st16(taddr, r);
        ptx::tmem_st16(taddr + 16, r + 16);
    }
}
template <int NR>
__device__ __forceinline__ void tmem_ld_n(uint32_t taddr, uint32_t *o) {
    if constexpr (NR == 16) {
        ptx::tmem_ld16(taddr, o);
    } else {
        ptx::tmem_ld16(taddr, o);
        ptx::tmem_ld16(taddr + 16, o + 16);
    }
}

// Tensor-core register group (complex64, R bits): the group's fused unitary, stored as the
// real-embedded B operand at `bhi` (B_hi, then B_lo), is applied on tiles of 128 rows.  Every
// thread splits its row x into A_hi = x rounded to nearest TF32 and A_lo = x - A_hi (exact in
// FP32; the tensor cores read it truncated to TF32, an error of either sign since A_lo has
// either sign), writes both to its TMEM lane, and one thread issues
//     D[:, 0:2K]  = A_hi [B_hi | B_lo]      (K/8 MMAs, N = 2K)
//     D[:, 0:K]  += A_lo B_hi               (K/8 MMAs, N = K)
// with FP32 accumulation; the row's result is D[:, 0:K] + D[:, K:2K] = A_hi B_hi + A_lo B_hi +
// A_hi B_lo (3xTF32).  Stacking B_hi and B_lo along N makes 2K/8 MMAs per tile instead of 3K/8:
// an MMA of N <= 128 costs its issuing thread about the same time whatever N is.
// NB (1 or 2) tiles are in flight per group; `mbar[k]` signals buffer k's MMAs' completion.
//
// RENORM: callers that cannot restore the state's norm once per circuit set RENORM: for a group
// whose fused matrix is unitary (the int after the B operand is nonzero) each output row is
// rescaled to its input row's norm, as y <- y (1 + d) with d = (|x|^2 - |y|^2) / (2 |y|^2).
template <int R, int NC, bool RENORM = false, int NB = 2>
__device__ __forceinline__ bool run_segment_tc(uint32_t buf, uint32_t seg, uint32_t bhi, int ctid, const int *swz,
                                               int c, uint32_t tcol, int bar_id, uint64_t *mbar, uint32_t (&phase)[2],
                                               volatile int *abort_flag, const uint64_t *wait_ns) {
    using G = TcGeom<R>;
    constexpr int NA = G::NA, K = G::K;
    constexpr int CH = 8;  // amplitudes per TMEM access batch (16 columns): fewer live registers
    int po[R], pf[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int p = lds_s8(seg + j);
        po[j] = 1 << p;
        pf[j] = po[j] ^ swz[p];
    }
    // A thread's row in tile t is row t * NC + ctid: its low 5 bits (the lane) pick lane bits, the
    // next two (the warp in the group, NC = 128) the first two rest bits, and the bits above (t)
    // rest bits 2, 3, ...; the warp's part is folded in here, the tile's read per tile.
    static_assert(NC == 128, "a tile is 128 rows: 4 warps of 32");
    const int lane = ctid & 31, wg = ctid >> 5;
    int wbase = 0, wfb = 0;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int p = lds_s8(seg + 8 + j);
        if ((lane >> j) & 1) { wbase |= 1 << p; wfb ^= swz[p]; }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int p = lds_s8(seg + 16 + j);
        if ((wg >> j) & 1) { wbase |= 1 << p; wfb ^= swz[p]; }
    }
    const int flags = lds_s8(seg + 14);
    const int T = (1 << (c - R)) / NC;  // 128-row tiles per chunk
    const uint32_t lane_off = (uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16;  // this thread's TMEM lane
    constexpr uint32_t idesc_wide = ptx::idesc_tf32(128, 2 * K), idesc_narrow = ptx::idesc_tf32(128, K);

    // group base (natural and swizzled) of this thread's row in tile t
    auto row_base = [&](int t, int &base, int &sbase) {
        int bs = wbase, fb = wfb;
        for (int j = 0; (t >> j) != 0; ++j)
            if ((t >> j) & 1) {
                const int p = lds_s8(seg + 18 + j);
                bs |= 1 << p;
                fb ^= swz[p];
            }
        base = bs;
        sbase = bs ^ fb;
    };
    // byte steps between the group's amplitudes in Gray-code order (the natural and the
    // swizzled address are both linear in the group index over GF(2)), load and store side
    uint32_t ld_step[R], st_step[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        ld_step[j] = (uint32_t)((flags & 1) ? po[j] : pf[j]) << 3;
        st_step[j] = (uint32_t)((flags & 2) ? po[j] : pf[j]) << 3;
    }
    bool failed = false;
    const bool renorm = RENORM && lds_s32(bhi + G::B_BYTES) != 0;
    // tile t -> TMEM buffer k; returns the row base
    auto stage = [&](int t, int k, int &base, int &sbase, float &nrm) -> bool {
        row_base(t, base, sbase);
        nrm = 0.f;
        const uint32_t col = tcol + (uint32_t)k * G::COLS + lane_off;
        // byte offset inside the chunk (< chunk bytes: every step flips bits below 2^c * 8); the
        // buffer base is only 1 KiB aligned, so it is added after the XOR walk, never XORed
        uint32_t off = (uint32_t)((flags & 1) ? base : sbase) << 3;
#pragma unroll
        for (int h = 0; h < NA / CH; ++h) {
            // Gray steps [h CH, h CH + CH) visit the amplitudes [g CH, g CH + CH), g = gray(h)
            const int g = h ^ (h >> 1);
            uint32_t ahi[2 * CH], alo[2 * CH];
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                const int b = h * CH + q;
                if (b) off ^= ld_step[low_bit(b)];
                const int gidx = (b ^ (b >> 1)) - g * CH;  // Gray code: this amplitude's index in the batch
                float xr, xi;
                SM<float>::ld(buf + off, xr, xi);
                const uint32_t hr = tf32_round(xr), hi_ = tf32_round(xi);
                ahi[2 * gidx] = hr;
                ahi[2 * gidx + 1] = hi_;
                alo[2 * gidx] = __float_as_uint(xr - __uint_as_float(hr));
                alo[2 * gidx + 1] = __float_as_uint(xi - __uint_as_float(hi_));
                if (RENORM) nrm = fmaf(xr, xr, fmaf(xi, xi, nrm));
            }
            tmem_st_n<2 * CH>(col + (uint32_t)(2 * CH * g), ahi);
            tmem_st_n<2 * CH>(col + (uint32_t)(K + 2 * CH * g), alo);
        }
        ptx::tmem_wait_st();
        ptx::tc_fence_before();
        // every row of the tile is in TMEM; the barrier also tells the group whether any
        // thread's wait for an earlier tile expired
        if (ptx::named_bar_or(bar_id, NC, failed)) return false;
        if (ctid == 0) {
            ptx::tc_fence_after();
            const uint32_t a = tcol + (uint32_t)k * G::COLS, d = a + 2 * K;
            // step s reads B rows [8s, 8s + 8): 256 bytes on, i.e. 16 in the descriptor's address
            // field (shared addresses stay below 2^18, so the field never carries over)
            const uint64_t bd = ptx::smem_desc_kmajor(bhi, 128, G::SBO);
#pragma unroll
            for (int s = 0; s < G::KSTEPS; ++s) ptx::mma_tf32_ts(d, a + 8 * s, bd + 16 * s, idesc_wide, s > 0);
#pragma unroll
            for (int s = 0; s < G::KSTEPS; ++s) ptx::mma_tf32_ts(d, a + K + 8 * s, bd + 16 * s, idesc_narrow, 1);
            ptx::mma_commit(&mbar[k]);
        }
        return true;
    };
    // wait for buffer k's product and write the tile (row base `base`/`sbase`) back to the chunk
    // (after an expired wait the tile is garbage; the group stops at its next barrier)
    auto finish = [&](int k, int base, int sbase, float nrm) {
        if (!ptx::mbar_wait(&mbar[k], phase[k], *(volatile const uint64_t *)wait_ns)) {
            failed = true;
            *abort_flag = 1;
        }
        phase[k] ^= 1;
        ptx::tc_fence_after();
        const uint32_t dcol = tcol + (uint32_t)k * G::COLS + 2 * K + lane_off;
        float ny = 0.f, dsc = 0.f;
        if (RENORM && renorm) {
            // the row's output norm first (a second pass over TMEM), then the scale
#pragma unroll
            for (int h = 0; h < NA / CH; ++h) {
                uint32_t y0[2 * CH], y1[2 * CH];
                tmem_ld_n<2 * CH>(dcol + (uint32_t)(2 * CH * h), y0);
                tmem_ld_n<2 * CH>(dcol + (uint32_t)(K + 2 * CH * h), y1);
                ptx::tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 2 * CH; ++q) {
                    const float v = __uint_as_float(y0[q]) + __uint_as_float(y1[q]);
                    ny = fmaf(v, v, ny);
                }
            }
            dsc = ny > 0.f ? 0.5f * (nrm - ny) / ny : 0.f;
        }
        uint32_t off = (uint32_t)((flags & 2) ? base : sbase) << 3;
#pragma unroll
        for (int h = 0; h < NA / CH; ++h) {
            const int g = h ^ (h >> 1);
            uint32_t y0[2 * CH], y1[2 * CH];
            tmem_ld_n<2 * CH>(dcol + (uint32_t)(2 * CH * g), y0);
            tmem_ld_n<2 * CH>(dcol + (uint32_t)(K + 2 * CH * g), y1);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                const int b = h * CH + q;
                if (b) off ^= st_step[low_bit(b)];
                const int gidx = (b ^ (b >> 1)) - g * CH;
                float yr = __uint_as_float(y0[2 * gidx]) + __uint_as_float(y1[2 * gidx]);
                float yi = __uint_as_float(y0[2 * gidx + 1]) + __uint_as_float(y1[2 * gidx + 1]);
                if (RENORM && renorm) {
                    yr = fmaf(yr, dsc, yr);
                    yi = fmaf(yi, dsc, yi);
                }
                SM<float>::st(buf + off, yr, yi);
            }
        }
    };
    int pb, ps;
    float pn;
    if constexpr (NB == 2) {  // two tiles in flight: tile t is staged (and its MMAs issued) while tile t-1's run
        if (!stage(0, 0, pb, ps, pn)) return false;
        for (int t = 1; t < T; ++t) {
            int nb, ns;
            float nn;
            if (!stage(t, t & 1, nb, ns, nn)) return false;
            finish((t - 1) & 1, pb, ps, pn);
            pb = nb;
            ps = ns;
            pn = nn;
        }
        finish((T - 1) & 1, pb, ps, pn);
    } else {  // one tile buffer: tiles one after another
        for (int t = 0; t < T; ++t) {
            if (!stage(t, 0, pb, ps, pn)) return false;
            finish(0, pb, ps, pn);
        }
    }
    return !ptx::named_bar_or(bar_id, NC, failed);  // the group leaves together
}

}  // namespace
}  // namespace sv
