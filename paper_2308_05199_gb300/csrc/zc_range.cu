// zc_range.cu -- extremes of the input and the relative error bound.
//
// A value-range relative bound eb = rel * (max - min) needs one full read of
// the input before compression.  Each CTA reduces a grid-strided share with
// 16-byte loads, writes its partial extremes to a slot of the workspace, and
// the last CTA to finish (a wrapping completion counter) combines the slots
// and resolves the bound in FP64 into the control block, so the compressor
// reads it from device memory and nothing returns to the host.
#include <cfloat>

#include "zc_launch.h"

namespace zc {

struct Acc {
    float mn, mx;
    bool bad;
};

__device__ __forceinline__ void acc_one(Acc& a, float v)
{
    a.bad |= !isfinite(v);
    a.mn = fminf(a.mn, v);
    a.mx = fmaxf(a.mx, v);
}

template <typename TX>
__device__ __forceinline__ void acc_vec(Acc& a, const uint4 v)
{
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (sizeof(TX) == 4) {
            acc_one(a, __uint_as_float(w[k]));
        } else {
            acc_one(a, __uint_as_float(w[k] << 16));
            acc_one(a, __uint_as_float(w[k] & 0xffff0000u));
        }
    }
}

// A thread's grid-strided share of one segment: four independent 16-byte
// streaming loads (ld.global.cs) in flight per thread, then the scalar tail.
// Measured on 512 MiB: 6.1 TB/s with streaming loads at 3 to 6 CTAs per SM,
// 5.3-5.4 TB/s with __ldg or ld.global.cg.  The pass runs from the end of
// the segment to its start, so the last lines it reads are the first ones
// the compressor reads next.
template <typename TX>
__device__ __forceinline__ void range_seg(Acc& a, const void* p, unsigned long long n,
                                          unsigned long long gtid, unsigned long long gstride)
{
    constexpr int VEC = 16 / sizeof(TX);
    constexpr int UNR = 4;
    unsigned long long nvec = 0;
    if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
        nvec = n / VEC;
        const uint4* top = (const uint4*)p + (nvec ? nvec - 1 : 0);  // vector i is top[-i]
        unsigned long long i = gtid;
        for (; i + (UNR - 1) * gstride < nvec; i += UNR * gstride) {
            uint4 v[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) v[u] = __ldcs(top - (long long)(i + u * gstride));
#pragma unroll
            for (int u = 0; u < UNR; ++u) acc_vec<TX>(a, v[u]);
        }
        for (; i < nvec; i += gstride) acc_vec<TX>(a, __ldcs(top - (long long)i));
    }
    for (unsigned long long i = nvec * VEC + gtid; i < n; i += gstride) {
        const float v = sizeof(TX) == 4 ? __ldg((const float*)p + i)
                                        : bf16_to_f32(__ldg((const unsigned short*)p + i));
        acc_one(a, v);
    }
}

struct RangeSegs {
    unsigned long long cnt[RANGE_MAX_SEGS];
    const void* ptr[RANGE_MAX_SEGS];
};

// Combine the per-thread extremes; the last CTA resolves the bound.
__device__ void range_finish(const RangeLaunch& P, Acc a)
{
    __shared__ float smn[8], smx[8];
    __shared__ int sbad[8];
    __shared__ bool is_last;
    // CTA reduction
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off; off >>= 1) {
        a.mn = fminf(a.mn, __shfl_xor_sync(FULL, a.mn, off));
        a.mx = fmaxf(a.mx, __shfl_xor_sync(FULL, a.mx, off));
    }
    a.bad = __any_sync(FULL, a.bad);
    if (lane == 0) {
        smn[warp] = a.mn;
        smx[warp] = a.mx;
        sbad[warp] = a.bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float mn = FLT_MAX, mx = -FLT_MAX;
        bool bad = false;
        for (int w = 0; w < 8; ++w) {
            mn = fminf(mn, smn[w]);
            mx = fmaxf(mx, smx[w]);
            bad |= sbad[w] != 0;
        }
        P.partial[blockIdx.x] = bad ? make_float2(__int_as_float(0x7fc00000), 0.0f) : make_float2(mn, mx);
        __threadfence();
        is_last = atomicInc(&P.ctl->range_done, gridDim.x - 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    float mn = FLT_MAX, mx = -FLT_MAX;
    bool bad = false;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
        const float vx = *(volatile float*)&P.partial[i].x;
        const float vy = *(volatile float*)&P.partial[i].y;
        const float2 v = make_float2(vx, vy);
        bad |= isnan(v.x);
        mn = fminf(mn, v.x);
        mx = fmaxf(mx, v.y);
    }
    for (int off = 16; off; off >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(FULL, mn, off));
        mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, off));
    }
    bad = __any_sync(FULL, bad);
    if (lane == 0) {
        smn[warp] = mn;
        smx[warp] = mx;
        sbad[warp] = bad;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 0; w < 8; ++w) {
        mn = fminf(mn, smn[w]);
        mx = fmaxf(mx, smx[w]);
        bad |= sbad[w] != 0;
    }
    Ctl* c = P.ctl;
    if (P.total == 0) mn = mx = 0.0f;
    c->mn = mn;
    c->mx = mx;
    if (P.minmax_out) {
        P.minmax_out[0] = mn;
        P.minmax_out[1] = mx;
    }
    if (bad) {
        fail(c, ZC_ERR_NONFINITE, 0);
        c->eb_ok = 0u;
        return;
    }
    if (P.rel > 0.0) {
        double e;
        if (mx == mn) {
            const double m = fabs((double)mx);
            e = P.rel * (m > 1.0 ? m : 1.0);
        } else {
            e = P.rel * ((double)mx - (double)mn);
        }
        const float ebf = (float)e;
        const float two = __fadd_rn(ebf, ebf);
        if (is_normal(ebf) && ebf > 0.0f && isfinite(two)) {
            c->eb = ebf;
            c->two_eb = two;
            c->inv = (float)(0.5 / (double)ebf);
            c->eb_ok = 1u;
        } else {
            fail(c, ZC_ERR_ARG, 0);
            c->eb_ok = 0u;
        }
    }
}

template <typename TX>
__global__ void __launch_bounds__(256) k_range_one(const RangeLaunch P)
{
    grid_dep_launch();  // the compressor after it may be launched now (it waits for the bound)
    Acc a{FLT_MAX, -FLT_MAX, false};
    const unsigned long long gtid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long gstride = (unsigned long long)gridDim.x * blockDim.x;
    range_seg<TX>(a, P.one.x, P.one.n, gtid, gstride);
    range_finish(P, a);
}

template <typename TX>
__global__ void __launch_bounds__(256) k_range_multi(const RangeLaunch P, const RangeSegs S)
{
    grid_dep_launch();  // the scatter pack after it may be launched now (it waits for the bound)
    Acc a{FLT_MAX, -FLT_MAX, false};
    const unsigned long long gtid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long gstride = (unsigned long long)gridDim.x * blockDim.x;
    // last segment first, each from its end: the first segment's start is read last
    for (unsigned k = P.n_segs; k-- > 0;) range_seg<TX>(a, S.ptr[k], S.cnt[k], gtid, gstride);
    range_finish(P, a);
}

__global__ void k_ws_init(Ctl* c)
{
    c->magic = WS_MAGIC;
}

cudaError_t launch_range(const RangeLaunch& R, unsigned grid, cudaStream_t s)
{
    if (R.dtype == ZC_F32) k_range_one<float><<<grid, 256, 0, s>>>(R);
    else k_range_one<uint16_t><<<grid, 256, 0, s>>>(R);
    return cudaGetLastError();
}

cudaError_t launch_range_multi(const RangeLaunch& R, const void* const* ptrs,
                               const unsigned long long* counts, unsigned nseg, unsigned grid,
                               cudaStream_t s)
{
    if (nseg > RANGE_MAX_SEGS) return cudaErrorInvalidValue;
    RangeSegs S;
    for (unsigned k = 0; k < nseg; ++k) {
        S.ptr[k] = ptrs[k];
        S.cnt[k] = counts[k];
    }
    RangeLaunch P = R;
    P.n_segs = nseg;
    if (R.dtype == ZC_F32) k_range_multi<float><<<grid, 256, 0, s>>>(P, S);
    else k_range_multi<uint16_t><<<grid, 256, 0, s>>>(P, S);
    return cudaGetLastError();
}

cudaError_t launch_ws_init(Ctl* ctl, cudaStream_t s)
{
    k_ws_init<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

}  // namespace zc
