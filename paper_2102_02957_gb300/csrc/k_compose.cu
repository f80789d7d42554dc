// Gate fusion for the tensor-core path: every register group of r bits (r = 3, 4, 5) in a
// blocking section becomes one dense 2^r x 2^r complex unitary, composed in FP64 on the GPU, then
// written as the B operand of a real GEMM in the tensor cores' canonical shared-memory layout,
// split into TF32 high and low parts.
//
// Real embedding: a register group holds NA = 2^r amplitudes x_c, stored interleaved as the row
// [re x_0, im x_0, re x_1, ...] (K = 2 NA).  The fused unitary U maps it to y_s = sum_c U_sc x_c,
// i.e. D = A B with
//     B[2c][2s] = Re U_sc,  B[2c+1][2s] = -Im U_sc,  B[2c][2s+1] = Im U_sc,  B[2c+1][2s+1] = Re U_sc.
// B (K rows x N = K columns) is stored K-major without swizzle: 8-row x 16-byte core matrices,
// element (k, n) at byte (n / 8) * SBO + (k / 4) * 128 + (n % 8) * 16 + (k % 4) * 4, SBO = 32 K;
// B_lo follows B_hi directly, so that the pair reads as one K x 2K operand [B_hi | B_lo].
// The high part is B rounded to TF32 (round to nearest), the low part the remainder, also
// rounded to nearest TF32 (the tensor cores would otherwise truncate it, a one-sided error).
#include "sv_internal.h"

namespace sv {
namespace {

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// One CTA per register group, thread j composes column j of U (U e_j through the group's gates).
template <int R>
__global__ void k_compose_f64(const ComposeSeg *__restrict__ segs, const DevGate<double> *__restrict__ gates,
                              unsigned char *__restrict__ prog, int *__restrict__ all_unitary) {
    constexpr int NA = 1 << R, K = 2 * NA, SBO = 32 * K;
    const ComposeSeg sg = segs[blockIdx.x];
    const int j = threadIdx.x;  // 0..NA-1
    double vr[NA], vi[NA];
    for (int b = 0; b < NA; ++b) { vr[b] = b == j ? 1.0 : 0.0; vi[b] = 0.0; }
    for (int gi = sg.g0; gi < sg.g1; ++gi) {
        const DevGate<double> &g = gates[gi];
        const int a = g.a;
        if (g.op == OP_DENSE1 || g.op == OP_DIAG1 || g.op == OP_X1) {
            double m[8];
            if (g.op != OP_DIAG1) {
                for (int k = 0; k < 8; ++k) m[k] = g.m[k];
            } else {
                m[0] = g.m[0]; m[1] = g.m[1]; m[2] = 0; m[3] = 0;
                m[4] = 0; m[5] = 0; m[6] = g.m[2]; m[7] = g.m[3];
            }
#pragma unroll
            for (int x = 0; x < NA; ++x) {
                if (x & (1 << a)) continue;
                const int y = x | (1 << a);
                const double ar = vr[x], ai = vi[x], br = vr[y], bi = vi[y];
                vr[x] = m[0] * ar - m[1] * ai + m[2] * br - m[3] * bi;
                vi[x] = m[0] * ai + m[1] * ar + m[2] * bi + m[3] * br;
                vr[y] = m[4] * ar - m[5] * ai + m[6] * br - m[7] * bi;
                vi[y] = m[4] * ai + m[5] * ar + m[6] * bi + m[7] * br;
            }
        } else {
            const int b = g.b;
            double m[32];
            for (int k = 0; k < 32; ++k) m[k] = 0.0;
            if (g.op == OP_DENSE2) {
                for (int k = 0; k < 32; ++k) m[k] = g.m[k];
            } else if (g.op == OP_DIAG2) {
                for (int r = 0; r < 4; ++r) { m[2 * (5 * r)] = g.m[2 * r]; m[2 * (5 * r) + 1] = g.m[2 * r + 1]; }
            } else {  // permutation: row r takes column m[r]
                for (int r = 0; r < 4; ++r) m[2 * (4 * r + (int)g.m[r])] = 1.0;
            }
#pragma unroll
            for (int x = 0; x < NA; ++x) {
                if (x & ((1 << a) | (1 << b))) continue;
                const int id[4] = {x, x | (1 << a), x | (1 << b), x | (1 << a) | (1 << b)};
                double xr[4], xi[4];
                for (int k = 0; k < 4; ++k) { xr[k] = vr[id[k]]; xi[k] = vi[id[k]]; }
                for (int r = 0; r < 4; ++r) {
                    double yr = 0, yi = 0;
                    for (int cc = 0; cc < 4; ++cc) {
                        const double mr = m[2 * (4 * r + cc)], mi = m[2 * (4 * r + cc) + 1];
                        yr += mr * xr[cc] - mi * xi[cc];
                        yi += mr * xi[cc] + mi * xr[cc];
                    }
                    vr[id[r]] = yr;
                    vi[id[r]] = yi;
                }
            }
        }
    }
    // unitarity of the fused matrix (in FP64): max |(U^H U - I)_ij| over all i, j
    __shared__ double ur[NA][NA + 1], ui[NA][NA + 1];
    __shared__ unsigned long long dev_bits;
    if (j == 0) dev_bits = 0;
    for (int r = 0; r < NA; ++r) { ur[r][j] = vr[r]; ui[r][j] = vi[r]; }
    __syncthreads();
    double worst = 0.0;
    for (int i = 0; i < NA; ++i) {
        double gr = 0.0, gi = 0.0;  // <U e_i, U e_j>
        for (int r = 0; r < NA; ++r) {
            gr += ur[r][i] * ur[r][j] + ui[r][i] * ui[r][j];
            gi += ur[r][i] * ui[r][j] - ui[r][i] * ur[r][j];
        }
        worst = fmax(worst, fabs(gr - (i == j ? 1.0 : 0.0)) + fabs(gi));
    }
    atomicMax(&dev_bits, (unsigned long long)__double_as_longlong(worst));  // non-negative: order as integers
    __syncthreads();
    const bool unitary = __longlong_as_double((long long)dev_bits) <= 1e-10;
    if (j == 0 && !unitary && all_unitary) atomicAnd(all_unitary, 0);
    if (j == 0 && sg.flag_off != kNoFlag) *reinterpret_cast<int *>(prog + sg.flag_off) = unitary ? 1 : 0;
    // column j of U is (vr, vi); write B entries with input index c = j
    unsigned char *bhi = prog + sg.b_off, *blo = bhi + 4 * K * K;
    auto b_offset = [](int k, int n) {
        return (uint32_t)((n >> 3) * SBO + (k >> 2) * 128 + (n & 7) * 16 + (k & 3) * 4);
    };
    for (int r = 0; r < NA; ++r) {
        const double u_re = vr[r], u_im = vi[r];
        const double val[4] = {u_re, -u_im, u_im, u_re};  // (k, n) = (2j, 2r), (2j+1, 2r), (2j, 2r+1), (2j+1, 2r+1)
        const int kk[4] = {2 * j, 2 * j + 1, 2 * j, 2 * j + 1};
        const int nn[4] = {2 * r, 2 * r, 2 * r + 1, 2 * r + 1};
        for (int e = 0; e < 4; ++e) {
            const float f = (float)val[e];
            const uint32_t hi = tf32_rna(f);
            const uint32_t lo = tf32_rna((float)(val[e] - (double)__uint_as_float(hi)));
            *reinterpret_cast<uint32_t *>(bhi + b_offset(kk[e], nn[e])) = hi;
            *reinterpret_cast<uint32_t *>(blo + b_offset(kk[e], nn[e])) = lo;
        }
    }
}

}  // namespace

void launch_compose(const void *dev_segs, int nseg, const void *dev_gates, void *dev_prog, int *all_unitary, int r,
                    cudaStream_t st) {
    if (nseg <= 0) return;
    const ComposeSeg *sg = (const ComposeSeg *)dev_segs;
    const DevGate<double> *g = (const DevGate<double> *)dev_gates;
    unsigned char *p = (unsigned char *)dev_prog;
    if (r == 3) k_compose_f64<3><<<nseg, 8, 0, st>>>(sg, g, p, all_unitary);
    else if (r == 4) k_compose_f64<4><<<nseg, 16, 0, st>>>(sg, g, p, all_unitary);
    else if (r == 5) k_compose_f64<5><<<nseg, 32, 0, st>>>(sg, g, p, all_unitary);
    else fail(SV_ERR_UNSUPPORTED, "fused groups have 3, 4 or 5 bits");
    check_cuda(cudaGetLastError(), "compose kernel launch");
}

}  // namespace sv
