// Tensor-core DFT of 16-point lines (sm_103a, tcgen05): the dense n-point
// DFT along one axis of the short-axis kernel written as a real GEMM
//   Y[line][2j + c'] = sum_{i, c} X[line][2i + c] G[2j + c'][2i + c]
// over interleaved (re, im) values, G the 32 x 32 real form of the complex
// matrix M = diag(post) F diag(pre) (F the DFT matrix of eq:F_defintion's
// discrete transform, pre and post the method's diagonal multipliers of that
// axis).  128 lines (one per thread of a warpgroup) form the A operand
// (M = 128 rows, K = 32), G the B operand (N = 32); the accumulator lives in
// tensor memory and comes back to the thread that owns the line.
//
// FP32 accuracy from lower-precision tensor-core inputs by split products,
// accumulated in FP32:
//  - TC_TF32X3: x = xb + xs and g = gb + gs with tf32 parts (round to
//    nearest), Y = Xb Gb + Xb Gs + Xs Gb (kind::tf32);
//  - TC_BF16X3: x = x1 + x2 + x3 and g = g1 + g2 + g3 with bfloat16 parts
//    (8 + 8 + 8 significant bits), Y = the six products X_a G_b with
//    a + b <= 4 (kind::f16, bf16 inputs).
//
// Operands sit in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, consecutive along K (LBO = 128 B),
// 8-row groups SBO bytes apart.  Every wait is bounded.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace mgk {
namespace {

enum { TC_NONE = 0, TC_TF32X3 = 1, TC_BF16X3 = 2 };

template <int TC> struct TcShape;
template <> struct TcShape<TC_TF32X3> {
  static constexpr int NSPLIT = 2;          // A and B parts in smem
  static constexpr int ESIZE = 4;           // bytes per element
  static constexpr int A_BYTES = 128 * 128; // 128 rows x 32 tf32
  static constexpr int B_BYTES = 32 * 128;  // 32 rows x 32 tf32
  static constexpr int SBO = 1024;          // 8 rows x 128 B
  static constexpr int KSTEP_BYTES = 256;   // K = 8 per instruction: 2 core matrices
  static constexpr int KSTEPS = 4;
  // kind::tf32: D f32 (bits 4-5 = 1), A and B tf32 (bits 7-9, 10-12 = 2),
  // K-major A and B, N >> 3 at bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
};
template <> struct TcShape<TC_BF16X3> {
  static constexpr int NSPLIT = 3;
  static constexpr int ESIZE = 2;
  static constexpr int A_BYTES = 128 * 64;  // 128 rows x 32 bf16
  static constexpr int B_BYTES = 32 * 64;
  static constexpr int SBO = 512;           // 8 rows x 64 B
  static constexpr int KSTEP_BYTES = 256;   // K = 16 per instruction: 2 core matrices
  static constexpr int KSTEPS = 2;
  // kind::f16 with bf16 A and B (format 1), D f32
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
};

constexpr int TC_TMEM_COLS = 64;  // 32 f32 accumulator columns per warpgroup, two warpgroups

// Byte offset of element (row, k) in a K-major operand of 32 elements per row.
template <int TC> __device__ __forceinline__ int tc_off(int row, int k) {
  constexpr int E = TcShape<TC>::ESIZE, PER = 16 / E;  // elements per 16-byte core-matrix row
  return (row >> 3) * TcShape<TC>::SBO + (k / PER) * 128 + (row & 7) * 16 + (k % PER) * E;
}

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29),
// SBO >> 4 (32-45), version 1 (bit 46), no swizzle (61-63 = 0).
template <int TC> __device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)((unsigned)TcShape<TC>::SBO >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t tc_f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Tensor-memory allocation of TC_TMEM_COLS columns by warp 0; the address is
// written to *slot.  Dealloc by warp 0 after every thread's last access.
// The .sync.aligned tcgen05 instructions need the whole warp converged at
// them: each is preceded by __syncwarp (the code before them can diverge,
// e.g. a bounded wait whose threads leave the loop at different polls).
__device__ __forceinline__ void tc_alloc(unsigned* slot) {
  __syncwarp();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
}
__device__ __forceinline__ void tc_dealloc(unsigned taddr) {
  __syncwarp();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_TMEM_COLS) : "memory");
}

__device__ __forceinline__ void tc_mma(int TC, uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  if (TC == TC_TF32X3)
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
  else
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive f32 columns of this thread's TMEM lane (row), warp w of the
// warpgroup reading lanes 32 (w % 4) .. 32 (w % 4) + 31.  The load and its
// wait are one asm statement: the destination registers of tcgen05.ld are
// undefined until tcgen05.wait::ld, and a separate statement would let the
// compiler copy or spill them in between.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Split value x (as FP64, exact for an FP32 input) into the parts of one
// operand element; parts[s] are the bit patterns stored in smem.
template <int TC> __device__ __forceinline__ void tc_split(double x, uint32_t* parts) {
  if (TC == TC_TF32X3) {
    const uint32_t b = tc_f32_to_tf32((float)x);
    parts[0] = b;
    parts[1] = tc_f32_to_tf32((float)(x - (double)__uint_as_float(b)));
  } else {
    double r = x;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const __nv_bfloat16 h = __float2bfloat16_rn((float)r);
      parts[s] = (uint32_t)__bfloat16_as_ushort(h);
      r -= (double)__bfloat162float(h);
    }
  }
}

// Write this thread's line (16 complex FP32 values) as row `row` of the A
// operand parts at `abase` (NSPLIT tiles of A_BYTES).
template <int TC> __device__ __forceinline__ void tc_stage_line(unsigned char* abase, int row, const float2* x) {
  using S = TcShape<TC>;
  if (TC == TC_TF32X3) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {  // 16-byte chunk c: x[2c], x[2c+1]
      uint32_t b[4], s[4];
      const float v[4] = {x[2 * c].x, x[2 * c].y, x[2 * c + 1].x, x[2 * c + 1].y};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        b[e] = tc_f32_to_tf32(v[e]);
        s[e] = tc_f32_to_tf32(v[e] - __uint_as_float(b[e]));
      }
      const int off = tc_off<TC>(row, 4 * c);
      *reinterpret_cast<uint4*>(abase + off) = make_uint4(b[0], b[1], b[2], b[3]);
      *reinterpret_cast<uint4*>(abase + S::A_BYTES + off) = make_uint4(s[0], s[1], s[2], s[3]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) {  // 16-byte chunk c: 8 bf16 = x[4c .. 4c+3]
      uint32_t w[3][4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 z = x[4 * c + e];
        float r0 = z.x, r1 = z.y;
        uint32_t p0[3], p1[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          const __nv_bfloat16 h0 = __float2bfloat16_rn(r0), h1 = __float2bfloat16_rn(r1);
          p0[s] = __bfloat16_as_ushort(h0);
          p1[s] = __bfloat16_as_ushort(h1);
          r0 -= __bfloat162float(h0);  // exact: the residual of an FP32 value
          r1 -= __bfloat162float(h1);
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) w[s][e] = p0[s] | (p1[s] << 16);
      }
      const int off = tc_off<TC>(row, 8 * c);
#pragma unroll
      for (int s = 0; s < 3; ++s)
        *reinterpret_cast<uint4*>(abase + s * S::A_BYTES + off) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
  }
}

// The B operand parts of one axis: the 32 x 32 real form of
// M[j][i] = post[j] W^{ji} pre[i], W = e^{-2 pi i/16} (e^{+2 pi i/16} for the
// inverse), pre and post = 1 when absent.  Work dealt over the CTA; the caller
// synchronises (and fences the async proxy) before the MMAs read it.
template <int TC, bool INV>
__device__ void tc_build_b(unsigned char* bbase, const float2* pre, const float2* post) {
  using S = TcShape<TC>;
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    const int j = e >> 4, i = e & 15;
    double sw, cw;
    sincospi((INV ? 2.0 : -2.0) * (double)((j * i) & 15) / 16.0, &sw, &cw);
    // m = post_j * w * pre_i in FP64 from the FP32 multipliers
    const double pr = pre ? pre[i].x : 1.0, pi = pre ? pre[i].y : 0.0;
    double mr = cw * pr - sw * pi, mi = cw * pi + sw * pr;
    if (post) {
      const double qr = post[j].x, qi = post[j].y;
      const double tr = qr * mr - qi * mi;
      mi = qr * mi + qi * mr;
      mr = tr;
    }
    // B[2j + c'][2i + c]: (re, re) = mr, (re, im) = -mi, (im, re) = mi, (im, im) = mr
    const double val[4] = {mr, -mi, mi, mr};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = 2 * j + (q >> 1), k = 2 * i + (q & 1);
      uint32_t parts[3];
      tc_split<TC>(val[q], parts);
      const int off = tc_off<TC>(n, k);
#pragma unroll
      for (int s = 0; s < S::NSPLIT; ++s) {
        if (TC == TC_TF32X3) *reinterpret_cast<uint32_t*>(bbase + s * S::B_BYTES + off) = parts[s];
        else *reinterpret_cast<uint16_t*>(bbase + s * S::B_BYTES + off) = (uint16_t)parts[s];
      }
    }
  }
}

// The split products of one warpgroup's 128 lines into the TMEM columns at
// dtmem (issued by one thread, after tcgen05.fence::after_thread_sync; the
// caller commits).
template <int TC>
__device__ __forceinline__ void tc_issue_products(uint32_t dtmem, const unsigned char* abase,
                                                  const unsigned char* bbase) {
  using S = TcShape<TC>;
  const uint32_t a0 = smem_u32(abase), b0 = smem_u32(bbase);
  int first = 1;
  // (A part, B part) pairs whose combined order is kept
  constexpr int NP = TC == TC_TF32X3 ? 3 : 6;
  const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
  for (int ks = 0; ks < S::KSTEPS; ++ks)
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) {
      const uint64_t da = tc_desc<TC>(a0 + pa[pr] * S::A_BYTES + ks * S::KSTEP_BYTES);
      const uint64_t db = tc_desc<TC>(b0 + pb[pr] * S::B_BYTES + ks * S::KSTEP_BYTES);
      tc_mma(TC, dtmem, da, db, S::IDESC, first ? 0 : 1);
      first = 0;
    }
}

}  // namespace
}  // namespace mgk
