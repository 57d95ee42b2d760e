// D3Q19 FP32-deviation step as two passes per time step:
//
//  k_mu3d      mu = k^2 psi'(rho) - kappa lap rho (Eq. 16) for every node, once
//              (step3d_mu.cuh).
//  k_coll3d    grad mu, grad rho (Eq. 17-25) -> F (Eq. 12) -> BGK + EDM
//              (Eq. 1, 6, 8) -> push streaming, plus the next density, for
//              a tile of 32 columns x a band of 11 rows marching through z.
//  k_coll3d_corners  the next density of the tiles' corner nodes.
//
// Compared with evaluating mu inside the collision kernel (where the halo
// makes each CTA recompute it ~2.3 times per node and the recomputation
// dominates shared-memory traffic), the split costs one extra float read and
// write per node (168 instead of 160 bytes per lattice update) and removes
// the mu phase, one block barrier per plane and most shared-memory loads from
// the collision kernel.  In k_coll3d one warp owns one 32-wide row of the
// tile, one lane per node, so the stencil reads of a warp are contiguous
// (free of bank conflicts) and no lane recomputes a neighbouring tile's node.
//
// The next density of a node is the sum of the 19 populations pushed into it.
// A node inside its tile receives them all from its own CTA.  A node in an
// edge row of its band (or an edge column of its tile) receives some from the
// band above or below (or the tile to the left or right): the two CTAs each
// add their partial sum by an atomic addition onto a zero the mu pass wrote,
// and since 0 + a + b does not depend on the order of the additions, the
// result is the same bits on every run.  A corner node (edge row and edge
// column) receives populations from up to four CTAs: their partial sums are
// added as 64-bit fixed-point integers (exact, so again independent of order)
// into an accumulator per corner, which k_coll3d_corners turns into the
// float density after the pass and zeroes for the next one.
#pragma once
#include <cuda.h>  // CUtensorMap

#include "lbm_device.cuh"
#include "step3d.cuh"
#include "step3d_fast.cuh"
#include "step3d_mu.cuh"

namespace lbmd {

// ------------------------------------------------------------------ collision pass
constexpr int CX = 32, CY = 11;     // default collision tile: 32 columns (lanes) x 11 rows (warps)
constexpr int TXC = CX, TYC = CY;
constexpr int CNT = CX * CY;        // 352 threads
constexpr int FW = CX;              // staged population row: the tile's 32 columns
constexpr int COLL_FD = 1;          // field planes issued this many planes ahead (1 or 2)

// Field planes: the density deviation and mu of a node side by side (one
// float2, x = deviation, y = mu), copied in by two 4-byte copies per node, so
// that every stencil offset of the two gradients is one 8-byte shared load.
// Staged populations: one row of 32 floats per tile row and population
// (x0 of a tile is a multiple of 32, so with nx % 4 == 0 a row is eight
// 16-byte chunks).  With VEC a CTA whose tile lies inside the lattice stages
// them with one tensor copy (TMA) per plane: a 32 x 11 x 1 x 19 box of the
// populations viewed as a 4-D tensor (x, y, z, i) lands in exactly this
// layout; the buffers are 1 KB aligned for it.  A ragged last tile in x or a
// short last band in y takes 16-byte copies that wrap around the periodic
// seams instead (tensor boxes that cross the lattice edge were measured to
// make those CTAs several times slower).
//
// RY rows of the tile (one warp each: the rows of one band of RowBands) and NB staged planes of populations: the copies of plane
// z + NB - 1 are issued while plane z is collided, so NB - 1 planes are in
// flight per CTA.  The field ring holds the 2R + 1 planes of the stencil plus
// the NB - 1 in flight.
__host__ __device__ constexpr int pow2_at_least(int n) { return n <= 1 ? 1 : 2 * pow2_at_least((n + 1) / 2); }

template <int S, int RY_ = CY, int NB_ = 2, int FD_ = 1>
struct CollShape {
  static constexpr int R = Sch<S>::R;
  static constexpr int RY = RY_, TY = RY_, NT = CX * RY_, NB = NB_, FD = FD_;
  static_assert(NB >= 2 && NB <= 4, "two to four staged planes");
  static_assert(FD == 1 || (FD == 2 && NB == 2 && !Sch<S>::GF), "field planes one or two planes ahead");
  static constexpr int GW = CX + 2 * R, GH = RY + 2 * R;  // field region (tile + stencil halo)
  // ring of field planes: FD = 1, the stencil's 2R + 1 and the NB - 1 in
  // flight, rounded up to a power of two so that a slot is a mask; FD = 2, the
  // stencil's and two more (one landed or in flight, one being issued)
  static constexpr int NS = FD == 1 ? pow2_at_least(2 * R + NB) : 2 * R + 1 + FD;
  static constexpr int plane = GH * GW;                   // float2 per field plane
  static constexpr int FPL = RY * FW;                     // staged populations of one i
  static constexpr int fbuf = (19 * FPL + 255) / 256 * 256;  // buffer stride (floats), 1 KB multiple
  static constexpr unsigned box_bytes = 19u * FPL * 4u;       // one tensor copy
  // compact schemes (GF): per collided node the density deviation and the six
  // derivative values (grad mu, grad rho) of its own plane, one set per staged plane
  static constexpr int NG = 7;
  static constexpr size_t fields_bytes = Sch<S>::GF ? size_t(NB) * NG * NT * 4 : size_t(NS) * plane * 8;
  static constexpr size_t off_f = (fields_bytes + 1023) / 1024 * 1024;
  static constexpr size_t bytes = off_f + size_t(NB) * fbuf * 4;
  // OBS: the snapshot values of the collided plane, one per thread, staged
  // like the populations (one set per staged plane)
  static constexpr size_t off_snap = bytes;
  static constexpr size_t bytes_obs = bytes + size_t(NB) * NT * 4;
  // field nodes per plane, and per thread; 16-byte population chunks, and per thread
  static constexpr int DE = plane;
  static constexpr int KD = (DE + NT - 1) / NT;
  static constexpr int FCH = 19 * RY * (FW / 4);
  static constexpr int KF = (FCH + NT - 1) / NT;
  // resident CTAs per SM the launch bounds ask for: two when two fit in the
  // SM's 228 KB of shared memory (1 KB of it reserved per CTA)
  static constexpr int MINB = 2 * (bytes_obs + 2048) <= size_t(228) * 1024 ? 2 : 1;
};

// grad rho and grad mu of a line scheme together from the interleaved field
// planes (x: density deviation, y: mu): one 8-byte load per stencil value and
// two packed FMAs per offset pair, d = p - q (as -1 q + p, one rounding) and
// acc += g d, instead of four scalar instructions.
template <int S>
__device__ __forceinline__ void grad3d_pair(const float2* sdm, const int* base, int W, int cx, int cy,
                                            float2& gx, float2& gy, float2& gz) {
  constexpr int R = Sch<S>::R;
  const float2 m1 = make_float2(-1.f, -1.f);
  float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
  const int c = cy * W + cx;
  auto pr = [&](int o) { return sdm[o]; };
#pragma unroll
  for (int m = 1; m <= R; ++m) {
    const float2 g = make_float2(float(Sch<S>::g(m)), float(Sch<S>::g(m)));
    ax = __ffma2_rn(g, __ffma2_rn(m1, pr(base[R] + c - m), pr(base[R] + c + m)), ax);
    ay = __ffma2_rn(g, __ffma2_rn(m1, pr(base[R] + c - m * W), pr(base[R] + c + m * W)), ay);
    az = __ffma2_rn(g, __ffma2_rn(m1, pr(base[R - m] + c), pr(base[R + m] + c)), az);
  }
  gx = ax;
  gy = ay;
  gz = az;
}

// mbarrier helpers of the tensor-copy staging.  Waits are bounded: after about
// a second of polling the wait gives up (the caller records an error) instead
// of hanging the GPU.  A copy that did not complete in time may still be
// writing into the CTA's shared memory, so k_coll3d then issues no further
// copy and, before the CTA exits, its issuing thread waits once more (again
// bounded) for that copy; the march in between computes on whatever arrived,
// in a step already marked bad.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  for (int it = 0; it < (1 << 20); ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// S a compact scheme (GF): the derivatives come from the fields gmu and grho
// (component-major, N each) of the line solves; no stencil halo.
// VEC: 16-byte copies (nx % 4 == 0, 16-byte aligned fields and populations),
// and tensor copies of the populations for CTAs whose tile lies inside the
// lattice (tmf: the populations as a 4-D tensor (nx, ny, nz, 19), box
// (FW, RY, 1, 19)).
// OBS: also reduce the observables of the state being advanced (max |v| with
// v = u + F / (2 rho), max |u|, mass, max |rho - snap|) into aux.partials, one
// set per CTA, and overwrite snap with this state's density deviation.
// The CTA (blockIdx.x = tile of ColTiles(nx), blockIdx.y = band of
// RowBands(ny, RY)) collides and pushes the nodes of its tile and band and
// gathers their next density.  Interior nodes get every incoming population
// from the CTA and are stored.  Edge-row and edge-column nodes lack those from
// the neighbouring band or tile; the CTA sums, per target node, the
// populations that leave through its edges (row by row across a band edge,
// column by column across a tile edge) and both partial sums go into rout by
// atomic addition onto the zeroes the mu pass wrote there.  Corner nodes and
// the populations leaving through a tile's corners go, as fixed-point
// integers (v * qscale rounded), into the corner accumulators qc
// (k_coll3d_corners indexing); rout is not touched at corner nodes.
template <int S, bool TAU1, bool VEC, bool OBS, int RY_ = CY, int NB_ = 2, int FD_ = COLL_FD>
__global__ void __launch_bounds__(CX* RY_, (CollShape<S, RY_, NB_, FD_>::MINB)) k_coll3d(const KParams p, const float* __restrict__ fin,
                                                    float* __restrict__ fout, const float* __restrict__ rin,
                                                    const float* __restrict__ muf, float* __restrict__ rout,
                                                    const StepAux aux, const int zc, float* __restrict__ snap,
                                                    const __grid_constant__ CUtensorMap tmf,
                                                    const float* __restrict__ gmu, const float* __restrict__ grho,
                                                    unsigned long long* __restrict__ qc, const float qscale) {
  using L = Lattice<1>;
  using Sh = CollShape<S, RY_, NB_, FD_>;
  constexpr int Q = 19, R = Sh::R, GW = Sh::GW, NS = Sh::NS, FPL = Sh::FPL;
  constexpr int RY = Sh::RY, NT = Sh::NT, NB = Sh::NB, FD = Sh::FD;
  extern __shared__ __align__(1024) unsigned char smem_c3[];  // (own name: other kernels align theirs to 16)
  unsigned char* smem = smem_c3;
  __shared__ __align__(8) unsigned long long s_bar[NB];  // tensor copies: one mbarrier per buffer
  constexpr bool GF = Sch<S>::GF;
  float2* s_dm = reinterpret_cast<float2*>(smem);
  float* s_g = reinterpret_cast<float*>(smem);  // GF: [NB][NG][NT]
  float* s_f = reinterpret_cast<float*>(smem + Sh::off_f);
  float* s_snap = reinterpret_cast<float*>(smem + Sh::off_snap);  // OBS only

  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int N = int(p.n), NXY = nx * ny;
  const ColTiles tiles(nx);
  const RowBands bands(ny, RY);
  const int tb = blockIdx.x, bb = blockIdx.y;
  const int x0 = tiles.start(tb), y0 = bands.start(bb), z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, nz);
  const int VW = tiles.start(tb + 1) - x0, VH = bands.start(bb + 1) - y0;
  const int tid = threadIdx.x;
  const int cy = tid / CX, cx = tid - cy * CX;  // one warp per row, one lane per column
  const bool crow = cy < VH;                    // a row of the band (warp-uniform)
  const bool cnode = cx < VW && crow;           // a node of the tile
  const bool top = cy == 0, bot = cy == VH - 1;  // edge rows (VH >= 2: never both)
  const bool lft = cx == 0, rgt = cx == VW - 1;  // edge columns (VW >= 2: never both)
  const bool corner = (lft || rgt) && (top || bot);
  const int gx = cx < VW ? x0 + cx : x0, gy = cy < VH ? y0 + cy : y0;
  // the row beyond this warp's band edge, the columns beyond the tile's edges
  const int yo = top ? wrapn(y0 - 1, ny) : wrapn(y0 + VH, ny);
  const int xo = lft ? wrapn(x0 - 1, nx) : wrapn(x0 + VW, nx);
  // corner accumulators: plane z, band b, tile t, corner c (bit 0: last
  // column of the tile, bit 1: last row of the band)
  const int ntx = tiles.nt, nbd = bands.nb;
  const int tm = tb == 0 ? ntx - 1 : tb - 1, tp = tb == ntx - 1 ? 0 : tb + 1;
  const int bm = bb == 0 ? nbd - 1 : bb - 1, bp = bb == nbd - 1 ? 0 : bb + 1;
  auto qadd = [&](int z, int b, int t, int c, float v) {
    const long long k = (((long long)z * nbd + b) * ntx + t) * 4 + c;
    atomicAdd(qc + k, (unsigned long long)__float2ll_rn(v * qscale));
  };
  const float omega = float(p.omega), rref = float(p.rho_ref);
  const int pc_first = z0 - 1, pc_last = z1;
  // staging buffer (populations, GF derivatives, OBS snapshot) of plane pc
  auto bsel = [&](int pc) { return int(unsigned(pc - pc_first) % unsigned(NB)); };
  // tensor copies when the tile (32 columns, RY rows) lies inside the lattice
  // (and the staging buffers 128-byte aligned, as tensor copies require)
  const bool tcta = VEC && x0 + FW <= nx && y0 + RY <= ny && (smem_u32(s_f) & 127u) == 0 &&
                    ((Sh::fbuf * 4) & 127) == 0;
  if (tcta && tid == 0) {
#pragma unroll
    for (int b = 0; b < NB; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned bar_phase = 0;  // bit b: parity of the next completion of s_bar[b]
  // a wait ran out: later waits are skipped and no copy is issued after it
  // (the step is already marked bad); the copy awaited then is lost_bar/lost_par
  bool tma_lost = false;
  unsigned lost_bar = 0, lost_par = 0;

  // the x-y part of the global offset of each of this thread's field nodes
  // (fixed for the whole z march; the shared offset of node e is e) and, VEC,
  // of its population chunks (shared offset of chunk c: 4 c)
  int dofs[Sh::KD], fofs[VEC ? Sh::KF : 1];
#pragma unroll
  for (int k = 0; k < Sh::KD; ++k) {
    const int e = tid + k * NT;
    const int ry = e / GW, rx = e - ry * GW;
    dofs[k] = e < Sh::DE ? wrapn(y0 - R + ry, ny) * nx + wrapn(x0 - R + rx, nx) : 0;
  }
  if constexpr (VEC) {
#pragma unroll
    for (int k = 0; k < Sh::KF; ++k) {
      const int c = tid + k * NT, i = c / (RY * (FW / 4));  // population of chunk c
      const int r = c - i * (RY * FW / 4), ry = r / (FW / 4), j = r - ry * (FW / 4);
      fofs[k] = i * N + wrapn(y0 + ry, ny) * nx + wrapn(x0 + 4 * j, nx);
    }
  }

  // field planes q (density deviation and mu) -> ring slot; populations of
  // plane q - R (if collided) -> its staging buffer
  // the field plane q (density deviation and mu) into ring slot `slot`
  auto issue_fields = [&](int q, int slot) {
    if constexpr (!GF) {
      const int zo = wrapi(q, nz) * NXY;  // q in [z0 - 1 - R, z1 + R]: one period at most
      float2* dd = s_dm + slot * Sh::plane;
#pragma unroll
      for (int k = 0; k < Sh::KD; ++k) {
        const int e = tid + k * NT;
        if (e < Sh::DE) {
          cpa4(&dd[e].x, rin + zo + dofs[k]);
          cpa4(&dd[e].y, muf + zo + dofs[k]);
        }
      }
    }
  };
  // the populations of plane pc (and, GF, this node's derivatives; OBS, its
  // snapshot value) into the plane's staging buffer
  auto issue_plane = [&](int pc) {
    const int zf = wrapi(pc, nz) * NXY;
    const int pb = bsel(pc);
    float* fd = s_f + pb * Sh::fbuf;
    if constexpr (GF) {
      // this node's deviation and derivatives in plane pc
      if (cnode) {
        float* gd = s_g + pb * Sh::NG * NT + tid;
        const int o = zf + gy * nx + gx;
        cpa4(gd, rin + o);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          cpa4(gd + (1 + a) * NT, gmu + a * N + o);
          cpa4(gd + (4 + a) * NT, grho + a * N + o);
        }
      }
    }
    if constexpr (VEC) {
      if (tcta) {
        if (tid == 0 && !tma_lost) {
          // the buffer's previous contents were read and written through the
          // generic proxy before the barrier that precedes this call
          const unsigned bar = smem_u32(&s_bar[pb]);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(Sh::box_bytes)
                       : "memory");
          asm volatile(
              "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(fd)),
              "l"(reinterpret_cast<unsigned long long>(&tmf)), "r"(x0), "r"(y0), "r"(wrapi(pc, nz)),
              "r"(0), "r"(bar)
              : "memory");
        }
      } else {
#pragma unroll
        for (int k = 0; k < Sh::KF; ++k) {
          const int c = tid + k * NT;
          if (c < Sh::FCH) cpa16(fd + 4 * c, fin + zf + fofs[k]);
        }
      }
    } else {
      if (cnode) {
        const float* fs = fin + zf + gy * nx + gx;
        float* fo = fd + cy * FW + cx;
#pragma unroll
        for (int i = 0; i < Q; ++i) cpa4(fo + i * FPL, fs + i * N);
      }
    }
    if constexpr (OBS) {
      // the snapshot of this thread's node in plane pc (push planes only)
      if (cnode && pc >= z0 && pc < z1) cpa4(s_snap + pb * NT + tid, snap + pc * NXY + gy * nx + gx);
    }
  };
  auto ring = [&](int v) {  // a slot index in [-NS, 2 NS) into [0, NS)
    if constexpr ((NS & (NS - 1)) == 0) return v & (NS - 1);
    else return v < 0 ? v + NS : (v >= NS ? v - NS : v);
  };

  // prologue.  FD = 1: field planes pc_first - R .. pc_first + R + NB - 2 with
  // the populations of planes pc_first .. pc_first + NB - 2, one copy group per
  // plane.  FD = 2: the stencil's field planes (one group), the populations of
  // plane pc_first (one group), field plane pc_first + R + 1 (one group); every
  // plane then commits two groups, its next plane's populations and the field
  // plane two planes ahead, so that waiting for all but the latest group leaves
  // that field plane in flight.
  int slot = 0;  // ring slot of plane pc_first - R + (number issued)
  if constexpr (FD == 1) {
    for (int q = pc_first - R; q <= pc_first + R + NB - 2; ++q) {
      issue_fields(q, slot);
      if (q - R >= pc_first) issue_plane(q - R);
      cpa_commit();
      slot = ring(slot + 1);
    }
  } else {
    for (int q = pc_first - R; q <= pc_first + R; ++q) {
      issue_fields(q, slot);
      slot = ring(slot + 1);
    }
    cpa_commit();
    issue_plane(pc_first);
    cpa_commit();
    issue_fields(pc_first + R + 1, slot);
    slot = ring(slot + 1);
    cpa_commit();
  }
  int sc = R;  // ring slot of the collision plane
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;     // next density of this node, planes pc - 1 .. pc + 1
  float oacc0 = 0.f, oacc1 = 0.f, oacc2 = 0.f;  // edge rows: of the node beyond the band, planes pc - 1 .. pc + 1
  float cacc0 = 0.f, cacc1 = 0.f, cacc2 = 0.f;  // edge columns: of the node beyond the tile, planes pc - 1 .. pc + 1
  const int fme = cy * FW + cx;  // this node in a staged population plane
  float o_v2 = 0.f, o_u2 = 0.f, o_d = 0.f;  // OBS: running maxima (4 |v|^2, |u|^2, |rho - snap|)
  float o_m = 0.f;                           // OBS: sum of this thread's density deviations
  int o_n = 0;                               // OBS: nodes counted
  const int snap_xy = gy * nx + gx;  // OBS: this thread's node in a plane
  for (int pc = pc_first; pc <= pc_last; ++pc) {
    // FD = 1: one copy group per plane, the NB - 2 latest may still be in
    // flight; FD = 2: the latest group (a field plane) may
    cpa_wait_n<FD == 1 ? NB - 2 : 1>();
    if (tcta) {
      // this plane's tensor copy has landed (bounded wait; on time-out the
      // step is marked bad and the march goes on with whatever arrived)
      const int b = bsel(pc);
      if (!tma_lost && !mbar_wait_bounded(smem_u32(&s_bar[b]), (bar_phase >> b) & 1u)) {
        atomicMin(aux.bad_step, 0ull);
        tma_lost = true;
        lost_bar = smem_u32(&s_bar[b]);
        lost_par = (bar_phase >> b) & 1u;
      }
      bar_phase ^= 1u << b;
      // this thread's generic accesses to the other buffer (the previous
      // plane) precede the tensor copy issued into it after the barrier
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if constexpr (FD == 1) {
      if (pc + NB - 1 <= pc_last) {
        issue_fields(pc + R + NB - 1, slot);
        issue_plane(pc + NB - 1);
        slot = ring(slot + 1);
      }
      cpa_commit();  // (empty at the end: the wait above counts one group per plane)
    } else {
      if (pc + 1 <= pc_last) issue_plane(pc + 1);
      cpa_commit();
      if (pc + 2 <= pc_last) {
        issue_fields(pc + R + 2, slot);
        slot = ring(slot + 1);
      }
      cpa_commit();
    }
    const int fbi = bsel(pc);
    float* fb = s_f + fbi * Sh::fbuf;
    float own0 = 0.f, ownp = 0.f, ownm = 0.f;  // this node's incoming populations with e_y = 0
    const bool live = pc >= z0 && pc < z1;     // a plane of this chunk (not a z halo plane)
    if (crow) {
      // every lane of a band row collides (lanes past a ragged tile on staged
      // values that nothing reads back), so that the exchanges by shuffle see a
      // converged warp; shared-memory stores are masked by cnode, pushes by push
      int base[2 * R + 1];
#pragma unroll
      for (int d = -R; d <= R; ++d) base[d + R] = ring(sc + d) * Sh::plane;
      float fv[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) fv[i] = fb[i * FPL + fme];
      const int c = (cy + R) * GW + cx + R;
      const float* gq = s_g + fbi * Sh::NG * NT + tid;  // GF
      const float dsv = GF ? gq[0] : s_dm[base[R] + c].x;
      const float rc = rref + dsv;
      // momentum from the differences of opposite populations (e_{i+1} = -e_i
      // for odd i): nine subtractions, then each component sums five of them
      float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
      for (int i = 1; i < Q; i += 2) {
        const float d = fv[i] - fv[i + 1];
        if (L::ex(i) != 0) jx = L::ex(i) > 0 ? jx + d : jx - d;
        if (L::ey(i) != 0) jy = L::ey(i) > 0 ? jy + d : jy - d;
        if (L::ez(i) != 0) jz = L::ez(i) > 0 ? jz + d : jz - d;
      }
      const float irc = __fdividef(1.f, rc);
      const float ux = jx * irc, uy = jy * irc, uz = jz * irc;
      float2 g2x, g2y, g2z;
      if constexpr (GF) {
        g2x = make_float2(gq[4 * NT], gq[1 * NT]);
        g2y = make_float2(gq[5 * NT], gq[2 * NT]);
        g2z = make_float2(gq[6 * NT], gq[3 * NT]);
      } else {
        grad3d_pair<S>(s_dm, base, GW, cx + R, cy + R, g2x, g2y, g2z);
      }
      const float grx = g2x.x, gry = g2y.x, grz = g2z.x, gmx = g2x.y, gmy = g2y.y, gmz = g2z.y;
      const float Fx = -rc * gmx + grx * (1.f / 3.f), Fy = -rc * gmy + gry * (1.f / 3.f),
                  Fz = -rc * gmz + grz * (1.f / 3.f);
      const float vx = ux + Fx * irc, vy = uy + Fy * irc, vz = uz + Fz * irc;
      const bool push = cnode && live;
      if (push && !(rc > 0.f)) atomicMin(aux.bad_step, (unsigned long long)aux.t);
      if constexpr (OBS) {
        if (push) {
          // 2 (u + F / (2 rho)) = u + v: the running maximum holds 4 |v_obs|^2
          const float hx = ux + vx, hy = uy + vy, hz = uz + vz;
          o_v2 = fmaxf(o_v2, hx * hx + hy * hy + hz * hz);
          o_u2 = fmaxf(o_u2, ux * ux + uy * uy + uz * uz);
          // the staged snapshot value was copied in before this plane's
          // barrier; it is overwritten with this state's deviation
          o_d = fmaxf(o_d, fabsf(dsv - s_snap[fbi * NT + tid]));
          snap[pc * NXY + snap_xy] = dsv;  // push planes lie in [z0, z1): no wrap
          o_m += dsv;  // at most one z-chunk of deviations per thread: FP32 suffices
          ++o_n;
        }
      }
      // target of population i = own node + per-axis deltas (periodic wrap folded in)
      const int pz = wrapi(pc, nz);
      const int dxp = (gx + 1 < nx) ? 1 : 1 - nx, dxm = (gx > 0) ? -1 : nx - 1;
      const int dyp = (gy + 1 < ny) ? nx : nx - NXY, dym = (gy > 0) ? -nx : NXY - nx;
      const int dzp = (pz + 1 < nz) ? NXY : NXY - N, dzm = (pz > 0) ? -NXY : N - NXY;
      float* fo = fout + pz * NXY + gy * nx + gx;
      const float vv15 = 1.5f * (vx * vx + vy * vy + vz * vz);
      const float uu15 = 1.5f * (ux * ux + uy * uy + uz * uz);
      const float wd0 = float(L::w(0)) * dsv, wd1 = float(L::w(1)) * dsv, wd2 = float(L::w(7)) * dsv;
      const float wr0 = float(L::w(0)) * rc, wr1 = float(L::w(1)) * rc, wr2 = float(L::w(7)) * rc;
      auto post = [&](const int i) {  // post-collision population i of this node
        const float wd = i == 0 ? wd0 : (i < 7 ? wd1 : wd2);
        const float wr = i == 0 ? wr0 : (i < 7 ? wr1 : wr2);
        const float ev = edot<L>(i, vx, vy, vz);
        const float Av = i == 0 ? -vv15 : ev * (3.f + 4.5f * ev) - vv15;
        if constexpr (TAU1) {
          return wd + wr * Av;
        } else {
          const float eu = edot<L>(i, ux, uy, uz);
          const float Au = i == 0 ? -uu15 : eu * (3.f + 4.5f * eu) - uu15;
          return (1.f - omega) * fv[i] + omega * wd + wr * (omega * Au + Av - Au);
        }
      };
      {
        // all 19 post-collision values first; at tau = 1 the pairs (i, i + 1)
        // of opposite velocities (e_{i+1} = -e_i for odd i) share e_i . v and
        // are evaluated two at a time by packed FMAs
        float pst[Q];
        if constexpr (TAU1) {
          pst[0] = post(0);
#pragma unroll
          for (int i = 1; i < Q; i += 2) {
            const float ev = edot<L>(i, vx, vy, vz);
            const float wd = i < 7 ? wd1 : wd2, wr = i < 7 ? wr1 : wr2;
            const float2 E = make_float2(ev, ev);
            const float2 T = __ffma2_rn(make_float2(4.5f, 4.5f), E, make_float2(3.f, -3.f));
            const float2 A = __ffma2_rn(E, T, make_float2(-vv15, -vv15));
            const float2 P = __ffma2_rn(make_float2(wr, wr), A, make_float2(wd, wd));
            pst[i] = P.x;
            pst[i + 1] = P.y;
          }
        } else {
#pragma unroll
          for (int i = 0; i < Q; ++i) pst[i] = post(i);
        }
        // populations that stay in this x-y column are gathered from
        // registers; those moving along the row (e_y = 0, e_x != 0) reach a
        // lane of this warp, which takes them by shuffle, except across the
        // tile's edge columns (the lane they reach by the shuffle's wrap is
        // not their target: the edge lane sums them for the tile beyond,
        // cacc); in an edge row, those leaving the band are summed per target
        // column the same way (oacc); the others go through shared memory
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (L::ey(i) != 0) continue;
          float v = pst[i];
          if (L::ex(i) != 0) {
            v = __shfl_sync(0xffffffffu, pst[i], (cx - L::ex(i)) & 31);
            if ((L::ex(i) > 0 && lft) || (L::ex(i) < 0 && rgt)) v = 0.f;  // from the tile beyond
          }
          if (L::ez(i) < 0) ownm += v; else if (L::ez(i) == 0) own0 += v; else ownp += v;
        }
        if (lft || rgt) {
          // edge columns: the populations leaving the tile along the row
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            if (L::ey(i) != 0 || L::ex(i) == 0) continue;
            if (!((L::ex(i) < 0 && lft) || (L::ex(i) > 0 && rgt))) continue;
            if (L::ez(i) < 0) cacc0 += pst[i]; else if (L::ez(i) == 0) cacc1 += pst[i]; else cacc2 += pst[i];
          }
        }
        if (top || bot) {
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            if (!((L::ey(i) < 0 && top) || (L::ey(i) > 0 && bot))) continue;
            float v = pst[i];
            if (L::ex(i) != 0) {
              v = __shfl_sync(0xffffffffu, pst[i], (cx - L::ex(i)) & 31);
              if ((L::ex(i) > 0 && lft) || (L::ex(i) < 0 && rgt)) v = 0.f;  // across a tile corner
            }
            if (L::ez(i) < 0) oacc0 += v; else if (L::ez(i) == 0) oacc1 += v; else oacc2 += v;
          }
          // the in-plane diagonal population leaving through the tile's
          // corner goes to the corner node of the diagonal neighbour
          // (D3Q19: 7 = (1,1,0), 8 = (-1,-1,0), 9 = (1,-1,0), 10 = (-1,1,0))
          if ((lft || rgt) && cnode && live) {
            const float v = top ? (lft ? pst[8] : pst[9]) : (lft ? pst[10] : pst[7]);
            qadd(pc, top ? bm : bp, lft ? tm : tp, (lft ? 1 : 0) | (top ? 2 : 0), v);
          }
        }
        if (cnode) {
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            if (L::ey(i) == 0 || (L::ey(i) < 0 && top) || (L::ey(i) > 0 && bot)) continue;
            fb[i * FPL + fme] = pst[i];
          }
        }
        // Away from the periodic seams the target offset of population i is
        // i N + e_x + e_y nx + e_z nx ny for every thread: a warp none of whose
        // pushing nodes lies on a seam stores with these common offsets.
        const bool seam = push && (gx == 0 || gx == nx - 1 || gy == 0 || gy == ny - 1 || pz == 0 || pz == nz - 1);
        if (!__any_sync(0xffffffffu, seam)) {
#pragma unroll
          for (int i = 0; i < Q; ++i)
            if (push) fo[i * N + L::ex(i) + L::ey(i) * nx + L::ez(i) * NXY] = pst[i];
        } else {
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            if (push) {
              const int d = (L::ex(i) > 0 ? dxp : (L::ex(i) < 0 ? dxm : 0)) +
                            (L::ey(i) > 0 ? dyp : (L::ey(i) < 0 ? dym : 0)) +
                            (L::ez(i) > 0 ? dzp : (L::ez(i) < 0 ? dzm : 0));
              fo[i * N + d] = pst[i];
            }
          }
        }
      }
    }
    __syncthreads();
    // gather for the tile's own node of this thread
    if (cnode) {
      float s_m = ownm, s_0 = own0, s_p = ownp;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (L::ey(i) == 0) continue;  // own column and row movers are in the registers
        if ((L::ey(i) > 0 && top) || (L::ey(i) < 0 && bot)) continue;  // from the neighbouring band
        if ((L::ex(i) > 0 && lft) || (L::ex(i) < 0 && rgt)) continue;  // from the neighbouring tile
        const float v = fb[i * FPL + fme - L::ey(i) * FW - L::ex(i)];
        if (L::ez(i) < 0) s_m += v; else if (L::ez(i) == 0) s_0 += v; else s_p += v;
      }
      acc0 += s_m;
      acc1 += s_0;
      acc2 += s_p;
      if (lft || rgt) {
        // edge columns: the in-plane diagonals leaving the tile from the
        // rows above and below in this band, for the node beyond this row
        float cv = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (L::ey(i) == 0 || L::ex(i) == 0) continue;
          if (!((L::ex(i) < 0 && lft) || (L::ex(i) > 0 && rgt))) continue;
          if ((L::ey(i) > 0 && top) || (L::ey(i) < 0 && bot)) continue;  // from the band beyond: a corner's
          cv += fb[i * FPL + fme - L::ey(i) * FW];
        }
        cacc1 += cv;
      }
      const int zt = pc - 1;
      if (zt >= z0 && zt < z1) {
        const int ro = zt * NXY + (y0 + cy) * nx;
        if (corner) {
          qadd(zt, bb, tb, (rgt ? 1 : 0) | (bot ? 2 : 0), acc0);
        } else if (top || bot || lft || rgt) {
          atomicAdd(rout + ro + x0 + cx, acc0);  // completed by the neighbour's addition (positivity: the mu pass)
        } else {
          rout[ro + x0 + cx] = acc0;
          if (!(rref + acc0 > 0.f)) atomicMin(aux.bad_step, (unsigned long long)(aux.t + 1));
        }
        if (top || bot) {
          // the node beyond the band edge: a corner of that band at a tile edge
          if (lft || rgt) qadd(zt, top ? bm : bp, tb, (top ? 2 : 0) | (rgt ? 1 : 0), oacc0);
          else atomicAdd(rout + zt * NXY + yo * nx + x0 + cx, oacc0);
        }
        if (lft || rgt) {
          // the node beyond the tile edge: a corner of that tile in an edge row
          if (top || bot) qadd(zt, bb, lft ? tm : tp, (lft ? 1 : 0) | (bot ? 2 : 0), cacc0);
          else atomicAdd(rout + ro + xo, cacc0);
        }
      }
      acc0 = acc1;
      acc1 = acc2;
      acc2 = 0.f;
      oacc0 = oacc1;
      oacc1 = oacc2;
      oacc2 = 0.f;
      cacc0 = cacc1;
      cacc1 = cacc2;
      cacc2 = 0.f;
    }
    sc = ring(sc + 1);
  }
  // the issuing thread keeps the CTA (and its shared memory) alive until a
  // copy that missed its wait has landed, or a second bounded wait runs out
  if (tcta && tid == 0 && tma_lost) (void)mbar_wait_bounded(lost_bar, lost_par);
  if constexpr (OBS)
    block_obs_reduce<NT>(0.5 * sqrt(double(o_v2)), sqrt(double(o_u2)), double(o_n) * p.rho_ref + double(o_m), double(o_d),
                          aux.partials + 4 * (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
}

// The next density of the corner nodes of k_coll3d's tiles: accumulator k =
// ((z nb + b) nt + t) 4 + c (nt tiles of ColTiles(nx), nb bands of
// RowBands(ny, ry); corner c: bit 0 the tile's last column, bit 1 the band's
// last row) holds the node's density deviation times qscale as a 64-bit
// integer; it is written to rout as a float (one rounding), flagged in bad at
// step t1 when the density is not positive, and zeroed for the next pass.
__global__ void __launch_bounds__(256) k_coll3d_corners(const KParams p, int ry, unsigned long long* __restrict__ qc,
                                                        float* __restrict__ rout, const float inv_qscale,
                                                        unsigned long long* bad, long long t1) {
  const ColTiles tiles(p.nx);
  const RowBands bands(p.ny, ry);
  const long long n = 4LL * tiles.nt * bands.nb * p.nz;
  const float rref = float(p.rho_ref);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int c = int(k & 3);
    const long long r = k >> 2;
    const int t = int(r % tiles.nt);
    const long long r2 = r / tiles.nt;
    const int b = int(r2 % bands.nb), z = int(r2 / bands.nb);
    const int x = (c & 1) ? tiles.start(t + 1) - 1 : tiles.start(t);
    const int y = (c & 2) ? bands.start(b + 1) - 1 : bands.start(b);
    const long long q = (long long)qc[k];
    qc[k] = 0ull;
    const float v = __ll2float_rn(q) * inv_qscale;
    rout[(long long)z * p.nx * p.ny + (long long)y * p.nx + x] = v;
    if (!(rref + v > 0.f)) atomicMin(bad, (unsigned long long)t1);
  }
}

}  // namespace lbmd
