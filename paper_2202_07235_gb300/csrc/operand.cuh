// Operand form of compressed rings for the tensor-core scoring path.
//
// Step 1 of eq. (image_innerproduct_pm), X_hat(q) = 2 pi sum_h conj(a_h(q)) b_h(q),
// is evaluated as real products of the (re, im) components of the half
// spectrum q = 0..Q/2 (slot 0 packs Re a(0), Re a(Q/2), as in the FP32 layout).
// The components are stored rounded to 16-bit floats, one plane per term:
//   RSVD_BF16   hi = rn_bf16(x)                     (1 plane)
//   RSVD_FP16   hi = rn_fp16(x)                     (1 plane)
//   RSVD_BF16X3 hi = rn_bf16(x), lo = rn_bf16(x - hi)  (2 planes: hi, then lo)
//   RSVD_FP16X3 x_s = x 2^e, hi = rn_fp16(x_s), lo = rn_fp16(x_s - hi)  (2 planes),
//               e per operand row (object, translation) from the row's largest
//               component m: e = 14 - E with 2^(E-1) <= m < 2^E, clamped to
//               [-126, 126] (e = 0 for a zero row); after the planes, one FP32
//               factor 2^-e per row (row n T + t)
// with x the FP32 coefficient.
//
// Geometry (G = 32 column groups, g = Q/64 slots per group, G * g = Q/2):
//   slot s belongs to group s % 32 at position u = s / 32;
//   K = 2 * Hp * g components per (object row, group), k = u * 2 Hp + 2 h + c
//   (c = 0: re, 1: im), Hp = H rounded up so that K is a multiple of 16
//   (and to an even number at Q = 512; components of h >= H are zero);
//   128 rows per tile: IPT = 128 / T objects per tile, row (lane) = (n % IPT) * T + t;
//   a plane is [tile][group][k / 8][lane 0..127][k % 8]: each (tile, group)
//   block is the canonical no-swizzle K-major tensor-core operand image of a
//   128 x K matrix (core matrices of 8 lanes x 8 components), 128 * K * 2 bytes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "rsvd_internal.cuh"

namespace rsvd {

constexpr int kOpGroups = 32;
constexpr int kOpLanes = 128;

struct OperandLayout {
  int Q, T, H;
  int g;    // slots per group
  int Hp;   // padded number of components
  int K;    // components per (row, group)
  int KC;   // K / 8
  int IPT;  // objects per 128-row tile
  long long N;  // objects
  long long tiles;
  long long plane_elems;  // 16-bit elements per plane
};

inline bool is_operand_precision(int precision) {
  return precision == RSVD_BF16 || precision == RSVD_FP16 || precision == RSVD_BF16X3 || precision == RSVD_FP16X3;
}
inline bool is_split_precision(int precision) { return precision == RSVD_BF16X3 || precision == RSVD_FP16X3; }
inline int operand_planes(int precision) { return is_split_precision(precision) ? 2 : 1; }
// Byte offset of the row factors (RSVD_FP16X3) and the form's total size.
inline size_t operand_scale_offset(const OperandLayout& L, int precision) {
  return (size_t)operand_planes(precision) * (size_t)L.plane_elems * 2u;
}
inline size_t operand_bytes(const OperandLayout& L, int precision) {
  const size_t rows = precision == RSVD_FP16X3 ? (size_t)L.N * (size_t)L.T : 0u;
  return operand_scale_offset(L, precision) + (rows * 4u + 15u) / 16u * 16u;
}

// Layout of N objects x T translations; false if (Q, T, H) is outside the
// tensor-core path (Q in {128, 256, 512}, T <= 64, H <= 32).
inline bool make_operand_layout(long long N, int T, int H, int Q, OperandLayout* L) {
  if (!(Q == 128 || Q == 256 || Q == 512) || T < 1 || T > kMaxT || H < 1 || H > 32 || N < 1) return false;
  L->Q = Q;
  L->T = T;
  L->H = H;
  L->g = Q / 64;
  // K = 2 Hp g multiple of 16  <=>  Hp multiple of 8 / g; at Q = 512 Hp is
  // even, so that a group's K-steps split into two equal halves
  const int step = L->g >= 8 ? 2 : 8 / L->g;
  L->Hp = (H + step - 1) / step * step;
  L->K = 2 * L->Hp * L->g;
  L->KC = L->K / 8;
  L->IPT = kOpLanes / T;
  L->N = N;
  L->tiles = (N + L->IPT - 1) / L->IPT;
  L->plane_elems = L->tiles * kOpGroups * (long long)L->K * kOpLanes;
  return true;
}

// Element index (component c = 0; c = 1 follows it) of (object n, translation
// t, component h, slot s) within a plane.
__host__ __device__ __forceinline__ long long operand_index(const OperandLayout& L, long long n, int t, int h,
                                                            int s) {
  const long long tile = n / L.IPT;
  const int lane = (int)(n % L.IPT) * L.T + t;
  const int grp = s & (kOpGroups - 1), u = s / kOpGroups;
  const int k = u * 2 * L.Hp + 2 * h;
  return (((tile * kOpGroups + grp) * L.KC + (k >> 3)) * kOpLanes + lane) * 8 + (k & 7);
}

// Round (re, im) into the planes of `precision` at element index idx.
__device__ __forceinline__ void operand_put(uint16_t* planes, long long plane_elems, int precision, long long idx,
                                            float2 v) {
  uint32_t* hi = reinterpret_cast<uint32_t*>(planes + idx);
  if (precision == RSVD_FP16) {
    const __half2 h = __floats2half2_rn(v.x, v.y);
    *hi = *reinterpret_cast<const uint32_t*>(&h);
    return;
  }
  const __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
  *hi = *reinterpret_cast<const uint32_t*>(&b);
  if (precision == RSVD_BF16X3) {
    const float2 r = make_float2(v.x - __bfloat162float(b.x), v.y - __bfloat162float(b.y));  // exact
    const __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
    *reinterpret_cast<uint32_t*>(planes + plane_elems + idx) = *reinterpret_cast<const uint32_t*>(&l);
  }
}

// Packs FP32 compressed rings (layout of rsvd_compress with RSVD_FP32) into
// the operand form (planes, and the row factors of RSVD_FP16X3) (operand.cu).
RSVD_HIDDEN int launch_pack_operands(const float2* c32, long long N, const OperandLayout& L, int precision,
                                     uint16_t* out, cudaStream_t stream);

}  // namespace rsvd
