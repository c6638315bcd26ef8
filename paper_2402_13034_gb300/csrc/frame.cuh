// RIS frame and face accessors shared by the path search and the polarisation kernels: FP64 loads of
// packed vectors, the frame's centre and axes in FP64, element positions e_m = c + a_m t1 + b_m t2,
// the FP32 unit normal and complex permittivity eps_r - j sigma / (omega eps0) of a face, and the
// mirror image of a direction.
#pragma once

#include "internal.cuh"

namespace risrt {

__device__ __forceinline__ d3 ld3(const dv4& p) { return D3(p.x, p.y, p.z); }
__device__ __forceinline__ d3 ldv(const float4& p) { return D3((double)p.x, (double)p.y, (double)p.z); }

__device__ __forceinline__ d3 fr_c(const Frame& F) { return D3(F.c[0], F.c[1], F.c[2]); }
__device__ __forceinline__ d3 fr_t1(const Frame& F) { return D3(F.t1[0], F.t1[1], F.t1[2]); }
__device__ __forceinline__ d3 fr_t2(const Frame& F) { return D3(F.t2[0], F.t2[1], F.t2[2]); }
__device__ __forceinline__ d3 fr_n(const Frame& F) { return D3(F.n[0], F.n[1], F.n[2]); }

__device__ __forceinline__ d3 elem_pos(const Frame& F, float4 e)
{
    return fr_c(F) + fr_t1(F) * (double)e.x + fr_t2(F) * (double)e.y;
}

__device__ __forceinline__ float3 face_n32(const DeviceScene& S, int f)
{
    const float4 p = S.faces[f].plane32;
    return f3(p.x, p.y, p.z);
}
__device__ __forceinline__ float2 face_eps32(const DeviceScene& S, int f, const WaveD& wv)
{
    const float2 m = S.mats[S.faces[f].mat];
    return make_float2(m.x, -m.y * wv.inv_we);
}
__device__ __forceinline__ float3 mirror_dir_f(float3 v, float3 n) { return v - n * (2.f * dot(n, v)); }

}  // namespace risrt
