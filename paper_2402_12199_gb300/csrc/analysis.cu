// Structure and kinetics analyses of a running system (paper, Results: the
// pair correlation function g(r) of the centres of mass, the mean square
// displacement, and the mean square rotation of SI Sec. 5 with the
// orientational distance d(q1, q2) = 1 - <q1, q2>^2).
//
//   * g(r) counts: one thread per listed body pair; the centre distance and
//     its bin are formed in FP32 with explicitly rounded IEEE operations in a
//     fixed order (no contraction into FMAs), so a CPU replaying the same
//     FP32 operations decides every bin the same way.  Counts go through a
//     shared-memory histogram per block, then integer atomics (exact in any
//     order).
//   * MSD / MSR: per body in FP64 from the unwrapped centres (pos + image x
//     box, the image counters kept by the integrator) and the reference frame
//     stored by rb_set_reference; per-block partial sums, then one block sums
//     them in a fixed order (deterministic).
#include <cmath>

#include "rb_internal.cuh"

namespace rb {

constexpr int kGrMaxBins = 4096;

__global__ void k_gr_counts(const int2* __restrict__ pairs, const int* __restrict__ n_pairs_ptr,
                            const float4* __restrict__ pos, float3 L, float3 invL, float rmax2,
                            float scale, int n_bins, unsigned* __restrict__ counts) {
    __shared__ unsigned hist[kGrMaxBins];
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    const int n = *n_pairs_ptr;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int2 ij = pairs[t];
        const float4 a = pos[ij.x], b = pos[ij.y];
        float dx = __fsub_rn(b.x, a.x), dy = __fsub_rn(b.y, a.y), dz = __fsub_rn(b.z, a.z);
        dx = __fsub_rn(dx, __fmul_rn(L.x, rintf(__fmul_rn(dx, invL.x))));
        dy = __fsub_rn(dy, __fmul_rn(L.y, rintf(__fmul_rn(dy, invL.y))));
        dz = __fsub_rn(dz, __fmul_rn(L.z, rintf(__fmul_rn(dz, invL.z))));
        const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        if (r2 < rmax2) {
            int k = (int)__fmul_rn(__fsqrt_rn(r2), scale);
            if (k > n_bins - 1) k = n_bins - 1;
            atomicAdd(&hist[k], 1u);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x)
        if (hist[b]) atomicAdd(&counts[b], hist[b]);
}

// Per block: sums over its bodies of |r_unwrapped - r_ref|^2 and of
// 1 - <q_ref, q>^2, in FP64 (two values per block).
__global__ void k_msd_msr_part(int N, const float4* __restrict__ pos, const int4* __restrict__ img,
                               const float4* __restrict__ quat, const float4* __restrict__ rpos,
                               const int4* __restrict__ rimg, const float4* __restrict__ rquat,
                               double3 L, double* __restrict__ part) {
    __shared__ double s_d[8], s_r[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0, rr = 0.0;
    if (i < N) {
        const float4 p = pos[i], p0 = rpos[i];
        const int4 m = img[i], m0 = rimg[i];
        const double dx = ((double)p.x - p0.x) + (double)(m.x - m0.x) * L.x;
        const double dy = ((double)p.y - p0.y) + (double)(m.y - m0.y) * L.y;
        const double dz = ((double)p.z - p0.z) + (double)(m.z - m0.z) * L.z;
        d2 = dx * dx + dy * dy + dz * dz;
        const float4 q = quat[i], q0 = rquat[i];
        const double c = (double)q.x * q0.x + (double)q.y * q0.y + (double)q.z * q0.z +
                         (double)q.w * q0.w;
        rr = 1.0 - c * c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_d[threadIdx.x >> 5] = d2;
        s_r[threadIdx.x >> 5] = rr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s_d[w];
            b += s_r[w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_msd_msr_final(const double* __restrict__ part, int n_part, int N,
                                double* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < n_part; k += 32) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
        out[0] = a / N;
        out[1] = b / N;
    }
}

}  // namespace rb

using namespace rb;

extern "C" {

rb_status rb_set_reference(rb_system* s) {
    if (!s) return fail(RB_EINVAL, "null system");
    const size_t N = (size_t)s->N;
    const int nb = (int)((N + 255) / 256);
    if (!s->ref_pos) {
        cudaError_t e = cudaMalloc((void**)&s->ref_pos, sizeof(float4) * N);
        if (e == cudaSuccess) e = cudaMalloc((void**)&s->ref_quat, sizeof(float4) * N);
        if (e == cudaSuccess) e = cudaMalloc((void**)&s->ref_image, sizeof(int4) * N);
        if (e == cudaSuccess) e = cudaMalloc((void**)&s->ana_part, sizeof(double) * (2 * nb + 2));
        if (e != cudaSuccess) return cuda_fail(e, "analysis reference");
    }
    RB_CUDA(cudaMemcpyAsync(s->ref_pos, s->pos, sizeof(float4) * N, cudaMemcpyDeviceToDevice, s->stream));
    RB_CUDA(cudaMemcpyAsync(s->ref_quat, s->quat, sizeof(float4) * N, cudaMemcpyDeviceToDevice, s->stream));
    RB_CUDA(cudaMemcpyAsync(s->ref_image, s->image, sizeof(int4) * N, cudaMemcpyDeviceToDevice, s->stream));
    return RB_OK;
}

rb_status rb_msd_msr(rb_system* s, double* msd, double* msr) {
    if (!s) return fail(RB_EINVAL, "null system");
    if (!s->ref_pos) return fail(RB_EINVAL, "no reference frame: call rb_set_reference first");
    const int N = (int)s->N;
    const int nb = (N + 255) / 256;
    k_msd_msr_part<<<nb, 256, 0, s->stream>>>(N, s->pos, s->image, s->quat, s->ref_pos,
                                              s->ref_image, s->ref_quat,
                                              make_double3(s->box[0], s->box[1], s->box[2]),
                                              s->ana_part);
    k_msd_msr_final<<<1, 32, 0, s->stream>>>(s->ana_part, nb, N, s->ana_part + 2 * nb);
    RB_CUDA(cudaGetLastError());
    double out[2];
    RB_CUDA(cudaMemcpyAsync(out, s->ana_part + 2 * nb, sizeof(out), cudaMemcpyDeviceToHost, s->stream));
    RB_CUDA(cudaStreamSynchronize(s->stream));
    if (msd) *msd = out[0];
    if (msr) *msr = out[1];
    return RB_OK;
}

rb_status rb_get_images(const rb_system* s, int32_t* images_host) {
    if (!s || !images_host) return fail(RB_EINVAL, "null argument");
    RB_CUDA(cudaMemcpyAsync(images_host, s->image, sizeof(int4) * s->N, cudaMemcpyDeviceToHost,
                            s->stream));
    RB_CUDA(cudaStreamSynchronize(s->stream));
    return RB_OK;
}

rb_status rb_gr_counts(rb_system* s, float r_max, int32_t n_bins, uint32_t* counts) {
    if (!s || !counts) return fail(RB_EINVAL, "null argument");
    if (n_bins < 1 || n_bins > kGrMaxBins) return fail(RB_EINVAL, "n_bins must be in [1, 4096]");
    if (!(r_max > 0.f) || r_max > s->Rc)
        return fail(RB_EINVAL, "r_max must be in (0, Rc]: the pair list holds pairs within Rc");
    RB_TRY(build_pairs_async(s, false, false));  // current list (skin check)
    const float3 L = make_float3(s->box[0], s->box[1], s->box[2]);
    const float3 invL = make_float3(1.f / s->box[0], 1.f / s->box[1], 1.f / s->box[2]);
    const float scale = (float)n_bins / r_max;
    k_gr_counts<<<s->num_sms * 4, 256, 0, s->stream>>>(s->pl.pairs, s->pl.n_pairs, s->pos, L, invL,
                                                       r_max * r_max, scale, n_bins, counts);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

rb_status rb_gr_normalise(const rb_system* s, const uint32_t* counts_host, int32_t n_bins,
                          float r_max, int64_t n_frames, double* g_host) {
    if (!s || !counts_host || !g_host) return fail(RB_EINVAL, "null argument");
    if (n_bins < 1 || !(r_max > 0.f) || n_frames < 1) return fail(RB_EINVAL, "bad arguments");
    // ideal-gas pair count in the shell [r_k, r_k+1): N (N - 1) / 2 of the
    // pairs, each in the shell with probability (4 pi / 3)(r_k+1^3 - r_k^3) / V
    const double kPi = 3.14159265358979323846;
    const double V = (double)s->box[0] * s->box[1] * s->box[2];
    const double N = (double)s->N;
    const double w = (double)r_max / n_bins;
    for (int k = 0; k < n_bins; ++k) {
        const double r0 = k * w, r1 = (k + 1) * w;
        const double ideal = 0.5 * N * (N - 1.0) * (4.0 * kPi / 3.0) * (r1 * r1 * r1 - r0 * r0 * r0) / V;
        g_host[k] = (double)counts_host[k] / ((double)n_frames * ideal);
    }
    return RB_OK;
}

}  // extern "C"
