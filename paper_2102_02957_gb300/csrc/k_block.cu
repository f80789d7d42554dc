// Blocking section: one HBM sweep applies every gate of the section to every chunk
// (Sec. IV.C, Listing 4: "for all chunks: fetch chunk, apply each gate of the section, swap
// out").  On one GPU the chunk of 2^c amplitudes (physical bits 0..c-1, contiguous) is the
// unit staged from HBM into shared memory; the transpiler (Sec. IV.A) guarantees that every
// gate of the section acts on chunk bits only.
//
// Kernel organisation (persistent, warp-specialised):
//  * warp 0, lane 0 is the producer: it streams the CTA's chunks j = blockIdx.x + t*gridDim.x
//    into a ring of NBUF shared-memory buffers with 1-D bulk asynchronous copies (TMA engine)
//    completing on "full" mbarriers;
//  * the other NC threads are consumers: for each chunk they run the section's register
//    groups -- each thread loads the 2^SEG_BITS amplitudes of a group (bits listed in the
//    group) from shared memory into registers, applies all the group's gates there, and
//    stores them back -- then one consumer writes the chunk back with a bulk copy and, once
//    a write-back has finished reading shared memory, releases that buffer to the producer
//    through an "empty" mbarrier (with a ring of >= 3 buffers the release of buffer t waits
//    until chunk t+1 is written back, so the consumer never stalls on its own write-back).
// Every wait is bounded (globaltimer); on expiry the kernel records DEV_ERR_TIMEOUT in the
// error word and stops.
#include "ptx.cuh"
#include "sv_internal.h"

namespace sv {
namespace {

constexpr uint64_t kWaitLimitNs = 4000000000ull;  // 4 s
constexpr int kPiece = 16384;                      // bytes per bulk copy instruction

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

constexpr int R = SEG_BITS;
constexpr int NA = 1 << R;  // amplitudes per register group

__device__ __forceinline__ int insert0(int x, int p) { return ((x >> p) << (p + 1)) | (x & ((1 << p) - 1)); }

template <typename T>
__device__ __forceinline__ void cmul_acc(T &yr, T &yi, T mr, T mi, T xr, T xi) {
    yr = fma(mr, xr, yr);
    yr = fma(-mi, xi, yr);
    yi = fma(mr, xi, yi);
    yi = fma(mi, xr, yi);
}

template <typename T, int A>
__device__ __forceinline__ void ap_dense1(T (&r)[NA], T (&i)[NA], const T *__restrict__ m) {
    const T m0r = m[0], m0i = m[1], m1r = m[2], m1i = m[3], m2r = m[4], m2i = m[5], m3r = m[6], m3i = m[7];
#pragma unroll
    for (int x = 0; x < NA; ++x) {
        if (x & (1 << A)) continue;
        const int y = x | (1 << A);
        const T ar = r[x], ai = i[x], br = r[y], bi = i[y];
        T pr = 0, pi = 0, qr = 0, qi = 0;
        cmul_acc(pr, pi, m0r, m0i, ar, ai);
        cmul_acc(pr, pi, m1r, m1i, br, bi);
        cmul_acc(qr, qi, m2r, m2i, ar, ai);
        cmul_acc(qr, qi, m3r, m3i, br, bi);
        r[x] = pr; i[x] = pi; r[y] = qr; i[y] = qi;
    }
}

template <typename T, int A>
__device__ __forceinline__ void ap_diag1(T (&r)[NA], T (&i)[NA], const T *__restrict__ m) {
    const T d0r = m[0], d0i = m[1], d1r = m[2], d1i = m[3];
#pragma unroll
    for (int x = 0; x < NA; ++x) {
        const T dr = (x & (1 << A)) ? d1r : d0r, di = (x & (1 << A)) ? d1i : d0i;
        const T xr = r[x], xi = i[x];
        r[x] = fma(dr, xr, -di * xi);
        i[x] = fma(dr, xi, di * xr);
    }
}

template <typename T, int A, int B>
__device__ __forceinline__ void ap_dense2(T (&r)[NA], T (&i)[NA], const T *__restrict__ m) {
    T mm[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) mm[k] = m[k];
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

template <typename T, int A, int B>
__device__ __forceinline__ void ap_diag2(T (&r)[NA], T (&i)[NA], const T *__restrict__ m) {
    T d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] = m[k];
#pragma unroll
    for (int x = 0; x < NA; ++x) {
        const int l = ((x >> A) & 1) | (((x >> B) & 1) << 1);
        const T dr = d[2 * l], di = d[2 * l + 1];
        const T xr = r[x], xi = i[x];
        r[x] = fma(dr, xr, -di * xi);
        i[x] = fma(dr, xi, di * xr);
    }
}

template <typename T, int A, int B>
__device__ __forceinline__ void ap_perm2(T (&r)[NA], T (&i)[NA], const T *__restrict__ m) {
    const int p0 = (int)m[0], p1 = (int)m[1], p2 = (int)m[2], p3 = (int)m[3];
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

template <typename T>
__device__ __forceinline__ void apply_gate(const DevGate<T> *__restrict__ g, int op, int code, T (&r)[NA], T (&i)[NA]) {
    const T *m = g->m;
#define SV_1Q(A)                                   \
    case A:                                        \
        if (op == OP_DENSE1) ap_dense1<T, A>(r, i, m); \
        else ap_diag1<T, A>(r, i, m);              \
        break;
#define SV_2Q(A, B)                                          \
    case A * R + B:                                          \
        if (op == OP_DENSE2) ap_dense2<T, A, B>(r, i, m);    \
        else if (op == OP_DIAG2) ap_diag2<T, A, B>(r, i, m); \
        else ap_perm2<T, A, B>(r, i, m);                     \
        break;
    if (op == OP_DENSE1 || op == OP_DIAG1) {
        switch (code) { SV_1Q(0) SV_1Q(1) SV_1Q(2) SV_1Q(3) default: break; }
    } else {
        switch (code) { SV_2Q(0, 1) SV_2Q(0, 2) SV_2Q(0, 3) SV_2Q(1, 2) SV_2Q(1, 3) SV_2Q(2, 3) default: break; }
    }
#undef SV_1Q
#undef SV_2Q
}

// One register group over the chunk in shared memory.
template <typename T, int NC, int KU>
__device__ __forceinline__ void run_segment(typename V2<T>::type *buf, int c, const DevSeg &sg,
                                            const DevGate<T> *__restrict__ gates, int ctid) {
    using T2 = typename V2<T>::type;
    const int p0 = sg.pos[0], p1 = sg.pos[1], p2 = sg.pos[2], p3 = sg.pos[3];
    int off[NA];
#pragma unroll
    for (int b = 0; b < NA; ++b)
        off[b] = ((b & 1) << p0) | (((b >> 1) & 1) << p1) | (((b >> 2) & 1) << p2) | (((b >> 3) & 1) << p3);
    const int G = 1 << (c - R);
    for (int g0 = ctid; g0 < G; g0 += NC * KU) {
        T re[KU][NA], im[KU][NA];
        int base[KU];
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            const int g = g0 + u * NC;
            base[u] = insert0(insert0(insert0(insert0(g, p0), p1), p2), p3);
            if (g < G) {
#pragma unroll
                for (int b = 0; b < NA; ++b) {
                    const T2 v = buf[base[u] + off[b]];
                    re[u][b] = v.x;
                    im[u][b] = v.y;
                }
            }
        }
        for (int gi = sg.g0; gi < sg.g1; ++gi) {
            const DevGate<T> *g = gates + gi;
            const int op = g->op, code = g->code;
#pragma unroll
            for (int u = 0; u < KU; ++u) apply_gate<T>(g, op, code, re[u], im[u]);
        }
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            if (g0 + u * NC < G) {
#pragma unroll
                for (int b = 0; b < NA; ++b) {
                    T2 v;
                    v.x = re[u][b];
                    v.y = im[u][b];
                    buf[base[u] + off[b]] = v;
                }
            }
        }
    }
}

template <typename T, int NC, int KU>
__global__ void __launch_bounds__(NC + 32, 1)
    k_block(typename V2<T>::type *__restrict__ state, int c, int64_t nchunks, int nbuf,
            const DevSeg *__restrict__ segs, int nseg, const DevGate<T> *__restrict__ gates, int *err) {
    using T2 = typename V2<T>::type;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int chunk_amps = 1 << c;
    const uint32_t chunk_bytes = (uint32_t)chunk_amps * (uint32_t)sizeof(T2);
    T2 *bufs = reinterpret_cast<T2 *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)nbuf * chunk_bytes);
    uint64_t *empty = full + nbuf;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + nbuf);

    if (threadIdx.x == 0) {
        for (int s = 0; s < nbuf; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();

    const int64_t count = blockIdx.x < nchunks ? (nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (threadIdx.x < 32) {
        // ------------------------------------------------------------ producer
        if (threadIdx.x != 0) return;
        int64_t issued = 0;
        for (int64_t it = 0; it < count; ++it) {
            const int s = (int)(it % nbuf);
            if (it >= nbuf) {
                if (!ptx::mbar_wait(&empty[s], (uint32_t)((it / nbuf - 1) & 1), kWaitLimitNs) || *abort_flag) {
                    atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
                    *abort_flag = 1;
                    break;
                }
            }
            const int64_t j = blockIdx.x + it * gridDim.x;
            const unsigned char *src = reinterpret_cast<const unsigned char *>(state + j * chunk_amps);
            unsigned char *dst = reinterpret_cast<unsigned char *>(bufs + (size_t)s * chunk_amps);
            ptx::mbar_arrive_expect_tx(&full[s], chunk_bytes);
            for (uint32_t o = 0; o < chunk_bytes; o += kPiece) {
                const uint32_t b = chunk_bytes - o < (uint32_t)kPiece ? chunk_bytes - o : (uint32_t)kPiece;
                ptx::bulk_g2s(dst + o, src + o, b, &full[s]);
            }
            ++issued;
        }
        // do not leave while copies into this CTA's shared memory are still in flight
        for (int64_t it = issued > nbuf ? issued - nbuf : 0; it < issued; ++it)
            (void)ptx::mbar_wait(&full[it % nbuf], (uint32_t)((it / nbuf) & 1), kWaitLimitNs);
        return;
    }

    // -------------------------------------------------------------- consumers
    const int ctid = threadIdx.x - 32;
    for (int64_t it = 0; it < count; ++it) {
        const int s = (int)(it % nbuf);
        const int64_t j = blockIdx.x + it * gridDim.x;
        if (!ptx::mbar_wait(&full[s], (uint32_t)((it / nbuf) & 1), kWaitLimitNs)) {
            atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
            *abort_flag = 1;
        }
        ptx::named_bar_sync(1, NC);
        if (*abort_flag) break;
        T2 *buf = bufs + (size_t)s * chunk_amps;
        for (int si = 0; si < nseg; ++si) {
            const DevSeg sg = segs[si];
            run_segment<T, NC, KU>(buf, c, sg, gates, ctid);
            if (si == nseg - 1) ptx::fence_proxy_async_smem();
            ptx::named_bar_sync(1, NC);
        }
        if (nseg == 0) ptx::fence_proxy_async_smem();
        if (ctid == 0) {
            unsigned char *dstg = reinterpret_cast<unsigned char *>(state + j * chunk_amps);
            const unsigned char *srcs = reinterpret_cast<const unsigned char *>(buf);
            for (uint32_t o = 0; o < chunk_bytes; o += kPiece) {
                const uint32_t b = chunk_bytes - o < (uint32_t)kPiece ? chunk_bytes - o : (uint32_t)kPiece;
                ptx::bulk_s2g(dstg + o, srcs + o, b);
            }
            ptx::bulk_commit();
            if (nbuf >= 3) {
                // release the previous buffer once its write-back has read shared memory; the
                // third buffer keeps a load in flight meanwhile
                ptx::bulk_wait_read<1>();
                if (it >= 1) ptx::mbar_arrive(&empty[(it - 1) % nbuf]);
            } else {
                ptx::bulk_wait_read<0>();
                ptx::mbar_arrive(&empty[s]);
            }
        }
    }
    if (ctid == 0) ptx::bulk_wait<0>();
}

template <typename T, int NC, int KU>
void launch_typed(void *state, int n, int c, const void *segs, int nseg, const void *gates, int *err,
                  cudaStream_t st) {
    using T2 = typename V2<T>::type;
    const int ce = c < n ? c : n;
    const size_t chunk_bytes = (size_t(1) << ce) * sizeof(T2);
    const int64_t nchunks = int64_t(1) << (n - ce);
    const size_t extra = 2 * 8 * 4 + 16;  // barriers + abort flag (up to 4 buffers)
    int nbuf = 3;
    const size_t max_smem = 227 * 1024;
    while (nbuf > 1 && nbuf * chunk_bytes + extra > max_smem) --nbuf;
    const size_t smem = nbuf * chunk_bytes + extra;
    if (smem > max_smem) fail(SV_ERR_UNSUPPORTED, "chunk does not fit in shared memory");
    auto kern = k_block<T, NC, KU>;
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "cudaFuncSetAttribute(block)");
    int per_sm = 0;
    check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NC + 32, smem), "occupancy(block)");
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(nchunks, (int64_t)num_sms() * per_sm);
    kern<<<(unsigned)grid, NC + 32, smem, st>>>((T2 *)state, ce, nchunks, nbuf, (const DevSeg *)segs, nseg,
                                                (const DevGate<T> *)gates, err);
    check_cuda(cudaGetLastError(), "block kernel launch");
}

}  // namespace

size_t devgate_bytes(int dtype) { return dtype == SV_C64 ? sizeof(DevGate<float>) : sizeof(DevGate<double>); }

void launch_block(int dtype, void *state, int n, int c, const void *dev_segs, int nseg, const void *dev_gates,
                  int ngates, int *dev_err, int threads, cudaStream_t st) {
    (void)ngates;
    (void)threads;
    const int ce = c < n ? c : n;
    if (ce < SEG_BITS) fail(SV_ERR_UNSUPPORTED, "blocked path needs a chunk of at least 4 bits");
    if (dtype == SV_C64)
        launch_typed<float, 256, 2>(state, n, c, dev_segs, nseg, dev_gates, dev_err, st);
    else
        launch_typed<double, 256, 1>(state, n, c, dev_segs, nseg, dev_gates, dev_err, st);
}

}  // namespace sv
