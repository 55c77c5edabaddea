// One RK stage of the nodal DG Maxwell operator, fused in a single kernel
// (FP32, CUDA cores).  Included by stage_n<N>.cu, one translation unit per order.
//
// Per tile of E consecutive tetrahedra (one CTA, persistent over tiles):
//   1. stage the six fields u[c][k][0..Np) and the 128-byte geometry records of
//      the tile in shared memory (coalesced loads);
//   2. flux extraction (Alg. 3 of the paper): for every face node, u- from the
//      tile, u+ from the tile when the neighbour is in it and from global
//      memory otherwise (PEC ghost on walls, zero on absorbing faces), the
//      upwind flux of Section 6 scaled by Fscale/2 (with materials: by Fscale
//      and the impedance coefficients of the face), into a shared flux tile
//      [6][E][4 Nfp];
//   3. local differentiation (Alg. 4): U_r, U_s, U_t = Dr U, Ds U, Dt U for
//      three fields at a time, chain rule with the element's metric terms
//      (Eq. dg-reference-matrices) and the curl (Eq. maxwells-claws),
//      accumulated in registers;
//   4. flux lifting (Alg. 1): rhs += LIFT * flux;
//   5. epilogue: either rhs -> global, or the LSERK4 update
//      res <- a res + dt rhs, u_out <- u + b res, so rhs never reaches HBM.
// The operator reads u_in and writes u_out (a different buffer): neighbours
// read u_in's face values during the same launch.
//
// Thread mapping: thread t = e + E*g handles element e of the tile and the
// rows (nodes) i = g + G*q, q < R, of the volume and lifting products.  With
// E = 32 every warp shares one g, so the matrix rows it reads are warp-uniform
// (one broadcast load per row); element-strided shared-memory rows use odd
// strides (no bank conflicts).
#pragma once

#include <cuda_runtime.h>

#include "device.h"
#include "launch.cuh"
#include "tcgen05.cuh"

namespace dgdev {

// Row groups G of the FP32 stage (a thread computes rows g, g + G, ... of the
// operator products): 2 (N = 3, 5, 6), 3 (N = 4, 7, 8) or 4 (N = 9) matrix rows
// per thread, measured fastest on GB300 (sweep meshes, ~1.7e7 DOFs: N = 4 with 7
// groups 476 us, 9 383, 12 343, 18 464; N = 6 with 21 groups 766, 28 730, 42 664;
// N = 7 with 30 groups 725, 40 714, 60 760; N = 9 with 44 groups 1256, 55 1252,
// 74 1317).
__host__ __device__ constexpr int fp32_row_groups(int N) {
  return N == 1 ? 4 : N == 2 ? 5 : N == 3 ? 10 : N == 4 ? 12 : N == 5 ? 28 : N == 6 ? 42 : N == 7 ? 40 : N == 8 ? 55 : 55;
}

template <int N, int S = 0> struct StageDims {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  static constexpr int E = stage_tile_elems(N, S), G = fp32_row_groups(N);
  static constexpr int T = E * G;
  static constexpr int R = (Np + G - 1) / G;
  static constexpr int US = Np | 1;                          // odd element stride
  static constexpr int FS = (Nfp % 2) ? NF : NF + 4;         // FS/4 odd: conflict-free float4
  static constexpr int UT = 6 * E * US;
  static constexpr int FT = 6 * E * (FS > US ? FS : US);     // flux tile, reused for rhs
  static constexpr int GT = E * kGeoWords;
  // orders 3..6: Dr/Ds/Dt (float4 rows) and LIFT staged in shared memory once
  // per CTA, next to the tile (they fit there; above N = 6 they are streamed or
  // read through L1).  N = 3, 4: with more row groups, 24 and 28 % faster than
  // reading them through L1; N = 1, 2 are faster through L1.
  static constexpr bool OPS_SMEM = N >= 3 && N <= 6;
  static constexpr int OT = OPS_SMEM ? 4 * Np * Np + Np * NF : 0;
  // orders 7, 8: Dr/Ds/Dt (230, 436 KB) are streamed through shared memory in
  // chunks of JC columns, two buffers: the copy of chunk c+1 (16-byte
  // asynchronous copies) runs while chunk c is multiplied (12 % faster than
  // reading them through L1; at N = 9 the chunks that fit, 11 columns, cost
  // more in barriers than they save, so N = 9 reads through L1)
  static constexpr bool OPS_STREAM = N == 7 || N == 8;
  static constexpr int JC = N == 7 ? 24 : 15;                 // divides Np
  static constexpr int NCH = (Np + JC - 1) / JC;
  // then LIFT in chunks of MC float4 columns (4 MC face nodes) through the same buffers
  static constexpr int MC = N == 7 ? 18 : 15;
  static constexpr int NLC = NF / 4 / MC;
  static constexpr int CT = OPS_STREAM ? 2 * 4 * Np * JC : 0;  // floats of the two chunk buffers
  static constexpr size_t smem_bytes = size_t(UT + FT + GT + OT + CT) * sizeof(float);
  // N = 4: keep two CTAs per SM (their shared tiles fit twice); without the
  // bound the asynchronous tile staging let it grow to 100 registers, one CTA
  // per SM and 440 us instead of 342.  Elsewhere 0 (no minimum): an explicit
  // minimum of 1 or 2 changed the register allocation at N = 1..3 (72 -> 134
  // registers at N = 1) and cost 10-50 %.
  static constexpr int MIN_CTAS = N == 4 ? 2 : 0;
  static_assert(smem_bytes <= 227 * 1024, "shared memory budget");
  static_assert((UT % 4) == 0 && (FT % 4) == 0 && (GT % 4) == 0, "tiles must stay 16-byte aligned");
  static_assert(!OPS_STREAM || (Np % JC == 0 && NF / 4 % MC == 0 && MC <= JC),
                "operator chunks tile the columns and fit the buffers");
};

// EXT: meshes with materials (A.mat) or absorbing faces; the vacuum
// instantiation compiles without any of that code.
template <int N, bool RK, bool EXT, int S>
__global__ void __launch_bounds__(StageDims<N, S>::T, StageDims<N, S>::MIN_CTAS) stage_kernel(const StageArgs A) {
  using D = StageDims<N, S>;
  constexpr int E = D::E, G = D::G, Np = D::Np, Nfp = D::Nfp, NF = D::NF, R = D::R;
  constexpr int US = D::US, FS = D::FS;
  extern __shared__ float4 smem4[];
  float* su = reinterpret_cast<float*>(smem4);
  float* sf = su + D::UT;
  float* sg = sf + D::FT;
  const float4* D4 = A.D4;
  const float4* LIFT4 = A.LIFT4;
  const int tid = threadIdx.x;
  pdl_launch_dependents();
  if constexpr (D::OPS_SMEM) {
    float4* sops = reinterpret_cast<float4*>(sg + D::GT);
    for (int i = tid; i < Np * Np; i += D::T) sops[i] = __ldg(A.D4 + i);
    for (int i = tid; i < Np * NF / 4; i += D::T) sops[Np * Np + i] = __ldg(A.LIFT4 + i);
    D4 = sops;
    LIFT4 = sops + Np * Np;
    // the first tile's __syncthreads (after its staging) publishes the copy
  }
  const int e = tid % E, g = tid / E;
  const int K = A.K;
  // orders 7, 8: a tile streams 2 NCH + NLC chunks, chunk gc into buffer gc & 1:
  // gc < 2 NCH columns [c JC, c JC + JC) of Dr/Ds/Dt (c = gc mod NCH, once per
  // pass), then LIFT columns [lc MC, lc MC + MC) of the float4 rows (lc = gc - 2 NCH)
  float4* cbuf = reinterpret_cast<float4*>(sg + D::GT + D::OT);
  auto issue_chunk = [&](int gc, int b) {
    if constexpr (D::OPS_STREAM) {
      float4* dst = cbuf + b * Np * D::JC;
      if (gc < 2 * D::NCH) {
        const int c = gc % D::NCH;
        for (int i = tid; i < Np * D::JC; i += D::T) {
          const int r = i / D::JC, jj = i - r * D::JC;
          tc::cp_async16(dst + i, A.D4 + r * Np + c * D::JC + jj);
        }
      } else {
        const int lc = gc - 2 * D::NCH;
        for (int i = tid; i < Np * D::MC; i += D::T) {
          const int r = i / D::MC, mm = i - r * D::MC;
          tc::cp_async16(dst + i, A.LIFT4 + r * (NF / 4) + lc * D::MC + mm);
        }
      }
      tc::cp_async_commit();
    }
  };
  pdl_wait();        // the previous kernel's fields are complete (operators are constant)

  for (int tt = blockIdx.x; tt < A.num_tiles; tt += gridDim.x) {
    const int tile = A.tile0 + tt;
    const int k0 = tile * E;
    const int Ev = min(E, K - k0);
    // the first operator chunk flies while the tile is staged and its fluxes formed
    // (buffer 0 was last read before the previous tile's final barriers)
    issue_chunk(0, 0);

    // ---- 1. stage geometry and fields (asynchronous copies, all in flight) --
    for (int idx = tid; idx < Ev * (kGeoWords / 4); idx += D::T)
      tc::cp_async16(reinterpret_cast<float4*>(sg) + idx, &A.geo[size_t(k0) * (kGeoWords / 4) + idx]);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float* src = A.u_in + (size_t(c) * K + k0) * Np;
      for (int idx = tid; idx < Ev * Np; idx += D::T) {
        const int ee = idx / Np, i = idx - ee * Np;
        tc::cp_async4(su + (c * E + ee) * US + i, src + idx);
      }
    }
    tc::cp_async_commit();
    tc::cp_async_wait_all();
    __syncthreads();

    // ---- 2. flux extraction -----------------------------------------------
    if (e < Ev) {
      const float* ge = sg + e * kGeoWords;
      const unsigned codes = __float_as_uint(ge[10]);
#pragma unroll
      for (int qm = 0; qm < (NF + G - 1) / G; ++qm) {
        const int m = g + G * qm;
        if (m >= NF) break;
        const int f = m / Nfp, j = m - f * Nfp;
        const int idM = __ldg(A.fmask + f * Nfp + j);
        float uM[6], uP[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) uM[c] = su[(c * E + e) * US + idM];
        const unsigned code = (codes >> (8 * f)) & 0xffu;
        if (code == 0u) {                       // perfectly conducting wall
#pragma unroll
          for (int c = 0; c < 3; ++c) { uP[c] = -uM[c]; uP[c + 3] = uM[c + 3]; }
        } else if (EXT && code == kAbsorbingCode) {   // characteristic absorbing: no incoming wave
#pragma unroll
          for (int c = 0; c < 6; ++c) uP[c] = 0.f;
        } else {
          const int k2 = __float_as_int(ge[28 + f]);
          const int i2 = __ldg(A.perm + (f * 24 + int(code) - 1) * Nfp + j);
          const int e2 = k2 - k0;
          if (e2 >= 0 && e2 < Ev) {
#pragma unroll
            for (int c = 0; c < 6; ++c) uP[c] = su[(c * E + e2) * US + i2];
          } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) uP[c] = __ldg(A.u_in + (size_t(c) * K + k2) * Np + i2);
          }
        }
        const float nx = ge[12 + 4 * f], ny = ge[13 + 4 * f], nz = ge[14 + 4 * f];
        const float sc = 0.5f * ge[15 + 4 * f];
        const float dEx = uM[0] - uP[0], dEy = uM[1] - uP[1], dEz = uM[2] - uP[2];
        const float dHx = uM[3] - uP[3], dHy = uM[4] - uP[4], dHz = uM[5] - uP[5];
        const float ndE = nx * dEx + ny * dEy + nz * dEz;
        const float ndH = nx * dHx + ny * dHy + nz * dHz;
        const float al = A.alpha;
        if (!EXT || !A.mat) {
          // E: -n x dH + alpha (n (n.dE) - dE);  H: n x dE + alpha (n (n.dH) - dH)
          const float fl[6] = {
              -(ny * dHz - nz * dHy) + al * (nx * ndE - dEx),
              -(nz * dHx - nx * dHz) + al * (ny * ndE - dEy),
              -(nx * dHy - ny * dHx) + al * (nz * ndE - dEz),
              (ny * dEz - nz * dEy) + al * (nx * ndH - dHx),
              (nz * dEx - nx * dEz) + al * (ny * ndH - dHy),
              (nx * dEy - ny * dEx) + al * (nz * ndH - dHz)};
#pragma unroll
          for (int c = 0; c < 6; ++c) sf[(c * E + e) * FS + m] = sc * fl[c];
        } else {
          // Section 6 with impedances: B_E (Z+ (-n x dH) + alpha (n (n.dE) - dE)),
          // B_H (Y+ (n x dE) + alpha (n (n.dH) - dH)), the coefficients of face f
          const float4 cf = __ldg(A.mat + size_t(k0 + e) * kMatVecs + 1 + f);
          const float fs = 2.f * sc, sE = fs * cf.y, sH = fs * cf.w;
          const float fl[6] = {
              cf.x * -(ny * dHz - nz * dHy) + al * (nx * ndE - dEx),
              cf.x * -(nz * dHx - nx * dHz) + al * (ny * ndE - dEy),
              cf.x * -(nx * dHy - ny * dHx) + al * (nz * ndE - dEz),
              cf.z * (ny * dEz - nz * dEy) + al * (nx * ndH - dHx),
              cf.z * (nz * dEx - nx * dEz) + al * (ny * ndH - dHy),
              cf.z * (nx * dEy - ny * dEx) + al * (nz * ndH - dHz)};
#pragma unroll
          for (int c = 0; c < 6; ++c) sf[(c * E + e) * FS + m] = (c < 3 ? sE : sH) * fl[c];
        }
      }
    }
    __syncthreads();

    // ---- 3. local differentiation and curl -------------------------------
    float rhs[6][R];
    int row[R];
#pragma unroll
    for (int q = 0; q < R; ++q) row[q] = min(g + G * q, Np - 1);
    {
      const float* ge = sg + e * kGeoWords;
      const float rx = ge[0], ry = ge[1], rz = ge[2];
      const float sx = ge[3], sy = ge[4], sz = ge[5];
      const float tx = ge[6], ty = ge[7], tz = ge[8];
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
        const int fb = pass == 0 ? 3 : 0;          // H fields first (curl H), then E
        const float* u0 = su + ((fb + 0) * E + e) * US;
        const float* u1 = su + ((fb + 1) * E + e) * US;
        const float* u2 = su + ((fb + 2) * E + e) * US;
        float acc[3][3][R];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int q = 0; q < R; ++q) acc[c][d][q] = 0.f;
        auto mac = [&](const float4& dm, int q, float v0, float v1, float v2) {
          acc[0][0][q] = fmaf(dm.x, v0, acc[0][0][q]);
          acc[0][1][q] = fmaf(dm.y, v0, acc[0][1][q]);
          acc[0][2][q] = fmaf(dm.z, v0, acc[0][2][q]);
          acc[1][0][q] = fmaf(dm.x, v1, acc[1][0][q]);
          acc[1][1][q] = fmaf(dm.y, v1, acc[1][1][q]);
          acc[1][2][q] = fmaf(dm.z, v1, acc[1][2][q]);
          acc[2][0][q] = fmaf(dm.x, v2, acc[2][0][q]);
          acc[2][1][q] = fmaf(dm.y, v2, acc[2][1][q]);
          acc[2][2][q] = fmaf(dm.z, v2, acc[2][2][q]);
        };
        if constexpr (D::OPS_STREAM) {
#pragma unroll 1
          for (int c = 0; c < D::NCH; ++c) {
            const int gc = pass * D::NCH + c;
            issue_chunk(gc + 1, (gc + 1) & 1);         // the next chunk (LIFT after the last)
            tc::cp_async_wait_group<1>();              // chunk gc has landed (this thread's)
            __syncthreads();                           // everyone's copies of chunk gc
            const float4* cb = cbuf + (gc & 1) * Np * D::JC;
#pragma unroll 4
            for (int jj = 0; jj < D::JC; ++jj) {
              const int j = c * D::JC + jj;
              const float v0 = u0[j], v1 = u1[j], v2 = u2[j];
#pragma unroll
              for (int q = 0; q < R; ++q) mac(cb[row[q] * D::JC + jj], q, v0, v1, v2);
            }
            __syncthreads();                           // buffer gc & 1 may be refilled
          }
        } else {
#pragma unroll 5
          for (int j = 0; j < Np; ++j) {
            const float v0 = u0[j], v1 = u1[j], v2 = u2[j];
#pragma unroll
            for (int q = 0; q < R; ++q)
              mac(D::OPS_SMEM ? D4[row[q] * Np + j] : __ldg(&A.D4[row[q] * Np + j]), q, v0, v1, v2);
          }
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
          float dx[3], dy[3], dz[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            dx[c] = rx * acc[c][0][q] + sx * acc[c][1][q] + tx * acc[c][2][q];
            dy[c] = ry * acc[c][0][q] + sy * acc[c][1][q] + ty * acc[c][2][q];
            dz[c] = rz * acc[c][0][q] + sz * acc[c][1][q] + tz * acc[c][2][q];
          }
          const float cx = dy[2] - dz[1], cy = dz[0] - dx[2], cz = dx[1] - dy[0];
          if (pass == 0) {        // dE/dt = curl H
            rhs[0][q] = cx; rhs[1][q] = cy; rhs[2][q] = cz;
          } else {                // dH/dt = -curl E
            rhs[3][q] = -cx; rhs[4][q] = -cy; rhs[5][q] = -cz;
          }
        }
      }
    }

    // ---- 4. lifting ------------------------------------------------------
    if constexpr (D::OPS_STREAM) {
      const float4* f4[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) f4[c] = reinterpret_cast<const float4*>(sf + (c * E + e) * FS);
#pragma unroll 1
      for (int lc = 0; lc < D::NLC; ++lc) {
        const int gc = 2 * D::NCH + lc;
        if (lc + 1 < D::NLC) {
          issue_chunk(gc + 1, (gc + 1) & 1);
          tc::cp_async_wait_group<1>();
        } else {
          tc::cp_async_wait_group<0>();
        }
        __syncthreads();
        const float4* cb = cbuf + (gc & 1) * Np * D::JC;
#pragma unroll 3
        for (int mm = 0; mm < D::MC; ++mm) {
          float4 fv[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) fv[c] = f4[c][lc * D::MC + mm];
#pragma unroll
          for (int q = 0; q < R; ++q) {
            const float4 L = cb[row[q] * D::MC + mm];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              float s = rhs[c][q];
              s = fmaf(L.x, fv[c].x, s);
              s = fmaf(L.y, fv[c].y, s);
              s = fmaf(L.z, fv[c].z, s);
              s = fmaf(L.w, fv[c].w, s);
              rhs[c][q] = s;
            }
          }
        }
        __syncthreads();
      }
    } else {
      const float4* f4[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) f4[c] = reinterpret_cast<const float4*>(sf + (c * E + e) * FS);
#pragma unroll 3
      for (int m4 = 0; m4 < NF / 4; ++m4) {
        float4 fv[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) fv[c] = f4[c][m4];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const float4 L = D::OPS_SMEM ? LIFT4[row[q] * (NF / 4) + m4]
                                       : __ldg(&A.LIFT4[row[q] * (NF / 4) + m4]);
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            float s = rhs[c][q];
            s = fmaf(L.x, fv[c].x, s);
            s = fmaf(L.y, fv[c].y, s);
            s = fmaf(L.z, fv[c].z, s);
            s = fmaf(L.w, fv[c].w, s);
            rhs[c][q] = s;
          }
        }
      }
    }
    __syncthreads();                         // flux tile no longer needed
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = g + G * q;
      if (i < Np && e < Ev) {
#pragma unroll
        for (int c = 0; c < 6; ++c) sf[(c * E + e) * US + i] = rhs[c][q];
      }
    }
    __syncthreads();

    // ---- 5. epilogue -----------------------------------------------------
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const size_t base = (size_t(c) * K + k0) * Np;
      for (int idx = tid; idx < Ev * Np; idx += D::T) {
        const int ee = idx / Np, i = idx - ee * Np;
        float r = sf[(c * E + ee) * US + i];
        if (EXT && A.mat) {                     // rhs_E / eps, rhs_H / mu
          const float4 w = __ldg(A.mat + size_t(k0 + ee) * kMatVecs);
          r *= c < 3 ? w.x : w.y;
        }
        if (RK) {
          const float dtk = A.dt_elem ? __ldg(A.dt_elem + k0 + ee) : A.dt;
          const float rn = fmaf(A.a, A.res[base + idx], dtk * r);
          A.res[base + idx] = rn;
          A.u_out[base + idx] = fmaf(A.b, rn, su[(c * E + ee) * US + i]);
        } else {
          A.rhs[base + idx] = r;
        }
      }
    }
    __syncthreads();
  }
}

template <int N, int S>
cudaError_t launch_stage_shape(bool rk, const StageArgs& a, int num_sms, cudaStream_t s) {
  using D = StageDims<N, S>;
  static int occ[2][2][16] = {};        // [rk][ext][device]: CTAs per SM
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  dev &= 15;
  const bool ext = a.mat || a.absorbing;
  auto kern = rk ? (ext ? stage_kernel<N, true, true, S> : stage_kernel<N, true, false, S>)
                 : (ext ? stage_kernel<N, false, true, S> : stage_kernel<N, false, false, S>);
  int& o = occ[rk ? 1 : 0][ext ? 1 : 0][dev];
  if (o == 0) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(D::smem_bytes));
    if (err != cudaSuccess) return err;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, D::T, D::smem_bytes);
    if (err != cudaSuccess) return err;
    if (o < 1) o = 1;
  }
  const int grid = a.num_tiles < num_sms * o ? a.num_tiles : num_sms * o;
  if (grid <= 0) return cudaSuccess;
  return launch_pdl(kern, grid, D::T, int(D::smem_bytes), s, a);
}

template <int N>
cudaError_t launch_stage_n(bool rk, const StageArgs& a, int num_sms, cudaStream_t s, int shape) {
  return shape == 1 ? launch_stage_shape<N, 1>(rk, a, num_sms, s)
                    : launch_stage_shape<N, 0>(rk, a, num_sms, s);
}

}  // namespace dgdev

#define DG_INSTANTIATE_STAGE(NN)                                                          \
  namespace dgdev {                                                                        \
  template cudaError_t launch_stage_n<NN>(bool, const StageArgs&, int, cudaStream_t, int); \
  }
