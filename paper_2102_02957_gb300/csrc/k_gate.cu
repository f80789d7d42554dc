// Per-gate path: one HBM sweep per gate (the paper's baseline, Sec. V.A; gate update of
// Sec. II.A).  A 1-qubit gate on qubit k updates every pair (i, i XOR 2^k) (Fig. 2); a 2-qubit
// gate every quadruple of indices that differ only in its two bits.
//
// Memory access: every thread moves whole 16-byte units.  For complex64 a unit holds the two
// amplitudes that differ in bit 0, so when bit 0 is not a gate qubit each unit carries two
// independent groups, and when it is, the unit holds both members of a pair.  For complex128
// a unit is one amplitude.  Consecutive threads take consecutive groups, so each warp reads
// and writes whole 128-byte lines.
#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 2;

__device__ __forceinline__ int64_t insert0(int64_t x, int p) {
    const int64_t low = x & ((int64_t(1) << p) - 1);
    return ((x >> p) << (p + 1)) | low;
}

template <typename T>
struct C2 { T re, im; };

template <typename T>
__device__ __forceinline__ void cmac(T &ore, T &oim, T mre, T mim, T xre, T xim) {
    ore = fma(mre, xre, ore);
    ore = fma(-mim, xim, ore);
    oim = fma(mre, xim, oim);
    oim = fma(mim, xre, oim);
}

template <typename T>
__device__ __forceinline__ void apply1(const T *m, T &x0r, T &x0i, T &x1r, T &x1i) {
    T y0r = 0, y0i = 0, y1r = 0, y1i = 0;
    cmac(y0r, y0i, m[0], m[1], x0r, x0i);
    cmac(y0r, y0i, m[2], m[3], x1r, x1i);
    cmac(y1r, y1i, m[4], m[5], x0r, x0i);
    cmac(y1r, y1i, m[6], m[7], x1r, x1i);
    x0r = y0r; x0i = y0i; x1r = y1r; x1i = y1i;
}

template <typename T>
__device__ __forceinline__ void apply2(const T *m, T (&xr)[4], T (&xi)[4]) {
    T yr[4], yi[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        yr[r] = 0; yi[r] = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac(yr[r], yi[r], m[2 * (4 * r + c)], m[2 * (4 * r + c) + 1], xr[c], xi[c]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) { xr[r] = yr[r]; xi[r] = yi[r]; }
}

// ---- complex64, 1 qubit, k >= 1: units u0, u1 = u0 | 2^(k-1) each hold two pairs' halves.
__global__ void __launch_bounds__(kThreads) k_gate1_c64_hi(float4 *a, int64_t groups, int kp, Mat1 M) {
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x;
    float4 A[kUnroll], B[kUnroll];
    int64_t u0[kUnroll];
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        const int64_t g = g0 + s * kThreads;
        u0[s] = insert0(g, kp);
        if (g < groups) { A[s] = a[u0[s]]; B[s] = a[u0[s] | (int64_t(1) << kp)]; }
    }
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        if (g0 + s * kThreads >= groups) continue;
        apply1(M.m, A[s].x, A[s].y, B[s].x, B[s].y);
        apply1(M.m, A[s].z, A[s].w, B[s].z, B[s].w);
        a[u0[s]] = A[s];
        a[u0[s] | (int64_t(1) << kp)] = B[s];
    }
}

// ---- complex64, 1 qubit, k == 0: each unit is one pair.
__global__ void __launch_bounds__(kThreads) k_gate1_c64_lo(float4 *a, int64_t units, Mat1 M) {
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x;
    float4 A[kUnroll];
#pragma unroll
    for (int s = 0; s < kUnroll; ++s)
        if (g0 + s * kThreads < units) A[s] = a[g0 + s * kThreads];
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        if (g0 + s * kThreads >= units) continue;
        apply1(M.m, A[s].x, A[s].y, A[s].z, A[s].w);
        a[g0 + s * kThreads] = A[s];
    }
}

// ---- complex64, 2 qubits, neither is qubit 0: 4 units per group, each unit two groups.
__global__ void __launch_bounds__(kThreads) k_gate2_c64_hi(float4 *a, int64_t groups, int p0, int p1, Mat2 M) {
    const int lo = p0 < p1 ? p0 : p1, hi = p0 < p1 ? p1 : p0;
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x;
    float4 U[kUnroll][4];
    int64_t base[kUnroll];
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        const int64_t g = g0 + s * kThreads;
        base[s] = insert0(insert0(g, lo), hi);
        if (g < groups) {
#pragma unroll
            for (int b = 0; b < 4; ++b)
                U[s][b] = a[base[s] | (int64_t(b & 1) << p0) | (int64_t(b >> 1) << p1)];
        }
    }
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        if (g0 + s * kThreads >= groups) continue;
        float xr[4], xi[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) { xr[b] = U[s][b].x; xi[b] = U[s][b].y; }
        apply2(M.m, xr, xi);
#pragma unroll
        for (int b = 0; b < 4; ++b) { U[s][b].x = xr[b]; U[s][b].y = xi[b]; xr[b] = U[s][b].z; xi[b] = U[s][b].w; }
        apply2(M.m, xr, xi);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            U[s][b].z = xr[b]; U[s][b].w = xi[b];
            a[base[s] | (int64_t(b & 1) << p0) | (int64_t(b >> 1) << p1)] = U[s][b];
        }
    }
}

// ---- complex64, 2 qubits, one of them is qubit 0: 2 units per group.  `zero_is_q0` says
// whether the gate's q[0] (low local bit) is qubit 0.
__global__ void __launch_bounds__(kThreads) k_gate2_c64_lo(float4 *a, int64_t groups, int po, int zero_is_q0, Mat2 M) {
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x;
    float4 U0[kUnroll], U1[kUnroll];
    int64_t base[kUnroll];
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        const int64_t g = g0 + s * kThreads;
        base[s] = insert0(g, po);
        if (g < groups) { U0[s] = a[base[s]]; U1[s] = a[base[s] | (int64_t(1) << po)]; }
    }
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        if (g0 + s * kThreads >= groups) continue;
        float xr[4], xi[4];
        if (zero_is_q0) {  // local b: bit0 -> element in unit, bit1 -> unit
            xr[0] = U0[s].x; xi[0] = U0[s].y; xr[1] = U0[s].z; xi[1] = U0[s].w;
            xr[2] = U1[s].x; xi[2] = U1[s].y; xr[3] = U1[s].z; xi[3] = U1[s].w;
        } else {           // local b: bit0 -> unit, bit1 -> element in unit
            xr[0] = U0[s].x; xi[0] = U0[s].y; xr[2] = U0[s].z; xi[2] = U0[s].w;
            xr[1] = U1[s].x; xi[1] = U1[s].y; xr[3] = U1[s].z; xi[3] = U1[s].w;
        }
        apply2(M.m, xr, xi);
        if (zero_is_q0) {
            U0[s] = make_float4(xr[0], xi[0], xr[1], xi[1]);
            U1[s] = make_float4(xr[2], xi[2], xr[3], xi[3]);
        } else {
            U0[s] = make_float4(xr[0], xi[0], xr[2], xi[2]);
            U1[s] = make_float4(xr[1], xi[1], xr[3], xi[3]);
        }
        a[base[s]] = U0[s];
        a[base[s] | (int64_t(1) << po)] = U1[s];
    }
}

// ---- complex128: one amplitude per 16-byte unit.
__global__ void __launch_bounds__(kThreads) k_gate1_c128(double2 *a, int64_t groups, int k, Mat1d M) {
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x;
    double2 A[kUnroll], B[kUnroll];
    int64_t i0[kUnroll];
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        const int64_t g = g0 + s * kThreads;
        i0[s] = insert0(g, k);
        if (g < groups) { A[s] = a[i0[s]]; B[s] = a[i0[s] | (int64_t(1) << k)]; }
    }
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        if (g0 + s * kThreads >= groups) continue;
        apply1(M.m, A[s].x, A[s].y, B[s].x, B[s].y);
        a[i0[s]] = A[s];
        a[i0[s] | (int64_t(1) << k)] = B[s];
    }
}

__global__ void __launch_bounds__(kThreads) k_gate2_c128(double2 *a, int64_t groups, int q0, int q1, Mat2d M) {
    const int lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
    const int64_t g0 = (int64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x;
    double2 U[kUnroll][4];
    int64_t base[kUnroll];
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        const int64_t g = g0 + s * kThreads;
        base[s] = insert0(insert0(g, lo), hi);
        if (g < groups) {
#pragma unroll
            for (int b = 0; b < 4; ++b) U[s][b] = a[base[s] | (int64_t(b & 1) << q0) | (int64_t(b >> 1) << q1)];
        }
    }
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
        if (g0 + s * kThreads >= groups) continue;
        double xr[4], xi[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) { xr[b] = U[s][b].x; xi[b] = U[s][b].y; }
        apply2(M.m, xr, xi);
#pragma unroll
        for (int b = 0; b < 4; ++b)
            a[base[s] | (int64_t(b & 1) << q0) | (int64_t(b >> 1) << q1)] = make_double2(xr[b], xi[b]);
    }
}

// complex64 with n == 1: the whole state is one unit.
__global__ void k_gate1_c64_single(float4 *a, Mat1 M) {
    float4 A = a[0];
    apply1(M.m, A.x, A.y, A.z, A.w);
    a[0] = A;
}

template <typename T>
__global__ void k_set_one(T *a, uint64_t idx) { a[idx] = T{1, 0}; }

inline unsigned grid_for(int64_t groups) {
    return (unsigned)((groups + (int64_t)kThreads * kUnroll - 1) / ((int64_t)kThreads * kUnroll));
}

}  // namespace

void launch_gate(int dtype, void *state, int n, const sv_gate &g, cudaStream_t st) {
    if (dtype == SV_C64) {
        float4 *a = (float4 *)state;
        if (g.nq == 1) {
            Mat1 M;
            for (int i = 0; i < 8; ++i) M.m[i] = (float)g.m[i];
            const int k = g.q[0];
            if (n == 1) {
                k_gate1_c64_single<<<1, 1, 0, st>>>(a, M);
            } else if (k == 0) {
                const int64_t units = int64_t(1) << (n - 1);
                k_gate1_c64_lo<<<grid_for(units), kThreads, 0, st>>>(a, units, M);
            } else {
                const int64_t groups = int64_t(1) << (n - 2);
                k_gate1_c64_hi<<<grid_for(groups), kThreads, 0, st>>>(a, groups, k - 1, M);
            }
        } else {
            Mat2 M;
            for (int i = 0; i < 32; ++i) M.m[i] = (float)g.m[i];
            const int q0 = g.q[0], q1 = g.q[1];
            if (q0 != 0 && q1 != 0) {
                const int64_t groups = int64_t(1) << (n - 3);
                k_gate2_c64_hi<<<grid_for(groups), kThreads, 0, st>>>(a, groups, q0 - 1, q1 - 1, M);
            } else {
                const int other = q0 == 0 ? q1 : q0;
                const int64_t groups = int64_t(1) << (n - 2);
                k_gate2_c64_lo<<<grid_for(groups), kThreads, 0, st>>>(a, groups, other - 1, q0 == 0 ? 1 : 0, M);
            }
        }
    } else {
        double2 *a = (double2 *)state;
        if (g.nq == 1) {
            Mat1d M;
            for (int i = 0; i < 8; ++i) M.m[i] = g.m[i];
            const int64_t groups = int64_t(1) << (n - 1);
            k_gate1_c128<<<grid_for(groups), kThreads, 0, st>>>(a, groups, g.q[0], M);
        } else {
            Mat2d M;
            for (int i = 0; i < 32; ++i) M.m[i] = g.m[i];
            const int64_t groups = int64_t(1) << (n - 2);
            k_gate2_c128<<<grid_for(groups), kThreads, 0, st>>>(a, groups, g.q[0], g.q[1], M);
        }
    }
    check_cuda(cudaGetLastError(), "per-gate kernel launch");
}

void launch_init_basis(int dtype, void *state, int n, uint64_t basis, cudaStream_t st) {
    const size_t bytes = (size_t(1) << n) * (dtype == SV_C64 ? 8 : 16);
    check_cuda(cudaMemsetAsync(state, 0, bytes, st), "cudaMemsetAsync");
    if (dtype == SV_C64)
        k_set_one<float2><<<1, 1, 0, st>>>((float2 *)state, basis);
    else
        k_set_one<double2><<<1, 1, 0, st>>>((double2 *)state, basis);
    check_cuda(cudaGetLastError(), "init kernel launch");
}

}  // namespace sv
