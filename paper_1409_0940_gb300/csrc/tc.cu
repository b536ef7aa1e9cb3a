// Tensor-core regeneration passes of the split-BF16 path (tcgen05 + TMA, sm_103a).
//
// One CTA owns a 128-row tile of operand A (data rows in pass 2 / prediction /
// materialisation; feature rows in pass 1) and walks a run of 128-row tiles of
// operand B (feature tiles, or data-row tiles).  For every B tile:
//
//   acc1 (TMEM, 128 x 128 fp32) = A_hi.B_hi^T + A_hi.B_lo^T + A_lo.B_hi^T     (X G, split BF16)
//   Z = sqrt(2/D) cos(acc1 + b)  -> Z_hi + Z_lo in shared memory            (the transform, Sec. 4)
//   acc2 (TMEM, 128 x m_pad fp32) += Z_hi.M_hi + Z_hi.M_lo + Z_lo.M_hi       (chained product)
//
// so that Z never reaches global memory (Sec. 3: Z_ij regenerated on the fly).
// acc2 is written out when a group of B tiles ends: per column block in pass 2
// (O'_ij = Z_ij W'_ij, eq. (gpOij)), once per split in pass 1 (Z_ij^T V_ij, the
// right-hand side of eq. (gpWij)), once for prediction.
//
// Warp roles (320 threads): warp 0 issues TMA loads, warp 1 owns TMEM and issues
// the MMAs (one thread), warps 2..9 run the epilogue (cos, split, stores); warps
// 2..5 take accumulator columns 0..63 and warps 6..9 columns 64..127, each warp
// the 32 TMEM lanes of its index mod 4.  acc1 is double-buffered so the cosine
// of tile t overlaps the products of tile t+1.  Every wait is bounded: on a
// timeout the CTA records an error code, stops issuing work, waits (bounded)
// for its own copies and products in flight, frees TMEM and returns.
//
// CTA pairs (CG = 2): a cluster of two CTAs owns two consecutive A tiles (256 rows) and
// walks the same B tiles.  The even CTA issues every MMA as tcgen05.mma.cta_group::2
// with M = 256: each CTA's shared memory holds its own 128 A rows and half of the B
// rows (64 of a B tile, m_pad/2 of a chained-operand chunk), and each CTA's tensor
// memory receives the accumulator rows of its own A tile.  Per MMA a CTA then reads
// 4 KB of A and 2 KB of B from shared memory instead of 4 + 4 KB, and its TMA ring
// fills 48 KB per 64-wide K chunk instead of 64 KB: shared-memory traffic, not the
// tensor pipe, bounds the single-CTA geometry (the N = 128 X.G product alone reads
// 128 bytes per clock at the tensor pipe's peak).  Both CTAs' copies complete on the
// even CTA's ring barriers, the MMA completions arrive on both CTAs' barriers
// (multicast commit), and the epilogue warps of both CTAs arrive on the even CTA's
// barriers.  The products and their order per output element are those of CG = 1,
// so results are bit-identical.  An A tile past the end of its row block (column block
// in pass 1, the query batch in scoring) is computed and discarded.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "tc.h"
#include "tcgen05.cuh"

namespace rff {

namespace {

constexpr int MODE_WRITEZ = 0, MODE_PASS1 = 1, MODE_PASS2 = 2, MODE_PREDICT = 3;
constexpr uint32_t ZBYTES = 65536;          // Z hi (32 KB) + Z lo (32 KB), two 64-column atoms each
constexpr uint32_t ZATOM = 16384;           // one 128 x 64 BF16 atom column of Z (128-byte rows)
constexpr int NEPI = 8;                     // epilogue warps
constexpr int NTHREADS = 64 + 32 * NEPI;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC2_COL = 256;         // acc2 with a single acc1 (ZT 0, 1)
constexpr int MAXG = 64;                    // groups (column blocks) per CTA
static_assert(COS_SCALE == 128.f, "the epilogues form COS_SCALE cos(.) as cos_rr_pow2<7>");
constexpr int PRED_GT = 8;                  // feature tiles per scoring group

// Ring geometry.  KC = K elements per ring stage: 64 (128-byte rows, 128-byte
// swizzle, 64 KB stages) or 32 (64-byte rows, 64-byte swizzle, 32 KB stages, so
// more stages fit beside the Z tile and more bytes are in flight).
//
// ZT selects where the Z tile lives between the cosine and the chained product:
// 0 = shared memory (128-byte swizzled K-major, the chained MMA reads it by
// descriptor), 1 = tensor memory (the chained MMA takes A from TMEM).  With Z in
// TMEM the shared memory it used holds more ring stages, and neither the Z stores
// nor the chained MMA's A reads use shared-memory bandwidth; acc1 is then single-
// buffered (TMEM: acc1 128 columns, Z hi 64, Z lo 64, acc2 at 256).  2 = Z in TMEM with
// acc1 double-buffered (acc1 at 0 and 128, Z hi 256, Z lo 320, acc2 at 384), for
// m_pad <= 128: the next X.G starts without waiting for the previous one to be read out.
// All issue the same products in the same order.
//
// CG = 2 runs the CTA pair (Z in TMEM only): a stage holds the CTA's A hi/lo (128 rows)
// and its half of B hi/lo (64 rows).
template <int KC, int ZT, int CG>
struct Ring {
  static_assert(CG == 1 || (CG == 2 && ZT != 0), "the CTA pair keeps Z in tensor memory");
  static constexpr uint32_t ROWB = KC * 2;               // bytes per operand row in a stage
  static constexpr uint32_t TILEB = 128 * ROWB;          // one 128-row operand tile
  static constexpr int BROWS = 128 / CG;                 // B rows of a tile held by this CTA
  static constexpr uint32_t BTILEB = BROWS * ROWB;       // this CTA's part of a B tile
  static constexpr uint32_t STAGEB = 2 * TILEB + 2 * BTILEB;   // A hi, A lo, B hi, B lo
  static constexpr int NS = CG == 2 ? ((KC == 64) ? 4 : 8)
                                    : (ZT ? ((KC == 64) ? 3 : 6) : ((KC == 64) ? 2 : 4));   // stages
  static constexpr int KSTEPS = KC / 16;                 // MMA K steps per stage
  static constexpr int CHUNKS = 128 / KC;                // chain-operand chunks per B tile
  static constexpr uint32_t LAYOUT = (KC == 64) ? 2 : 4; // descriptor layout: 128B / 64B swizzle
  static constexpr uint32_t SBO = 8 * ROWB;              // bytes between 8-row groups
  static constexpr uint32_t ZSMEM = ZT ? 0 : ZBYTES;     // shared memory of the Z tile
};
template <int KC, int ZT, int CG>
constexpr size_t smem_bytes();   // defined after Shared
// TMEM columns of Z hi (Z lo follows, 64 columns each) and of acc2 for each Z placement
__host__ __device__ constexpr uint32_t zh_col(int zt) { return zt == 2 ? 256 : 128; }
__host__ __device__ constexpr uint32_t acc2_col(int zt) { return zt == 2 ? 384 : ACC2_COL; }

// error codes written to the error word
constexpr int ERR_TIMEOUT_PRODUCER = 1, ERR_TIMEOUT_MMA = 2, ERR_TIMEOUT_EPI = 4;

struct TcArgs {
  CUtensorMap tA_hi, tA_lo, tB_hi, tB_lo, tM_hi, tM_lo;   // B and M boxes: 128/CG and m_pad/CG rows
  int mode, nk, mpad, R, C, nsplit;
  int64_t a_rows;                           // scoring: valid query rows (CTA pairs discard the rest)
  const float* bias;
  const int32_t* a_ok;
  const int32_t* b_ok;
  float scale;
  int64_t nrow_tiles;                       // pass 2: 128-row tiles of the data (work items x C)
  float inv_xg;                             // X.G accumulator -> X G (1 / (xscale gscale))
  const unsigned* m_amax;                   // max |M| of the chained operand (its FP16 split scale)
  unsigned* out_amax;                       // pass 2: receives max |out| (float bits), or null
  const int64_t* row_slot;
  const int64_t* row_size;
  const int64_t* col_slot;
  const int64_t* col_size;
  int64_t fslots;
  float* out;
  int64_t out_elems;                        // elements of out's layout (checked in bounds-checked builds)
  int64_t out_block_stride;
  int64_t wz_r0, wz_nr, wz_f0, wz_nf, ldo;  // materialisation window
  __half *zt_hi, *zt_lo;                    // write mode: Z^T as an FP16 hi/lo split (ld ldo), or null
  float zt_scale;                           // its power-of-two scale
  int bias_in_mma;                          // 1: b already in the product (column of ones)
  const uint8_t* bmask;                     // passes 1 and 2: active blocks (R x C), or null
  int m_shared;                             // pass 1: the chained operand's rows 0..m_pad serve every block
  int* err;
  long long timeout_cycles;
};

using namespace tc5;

// ------------------------------------------------------------------ shared state
template <int NS, int MG = MAXG>
struct Shared {
  static constexpr int maxg = MG;   // groups of B tiles a CTA may take
  uint64_t full[NS], empty[NS];
  uint64_t acc1_full[2], acc1_empty[2];
  uint64_t z_full, z_empty, acc2_full, acc2_empty, mma_done;
  uint32_t tmem_base;
  int abort_flag;
  int ngroups;
  int m_y;
  int64_t a_row0;
  int64_t g_b0[MG];
  int g_nt[MG];
  float* g_out[MG];
  int64_t g_arow[MG];     // A tile row of the group (pass 2 takes work items of several row tiles)
  int g_my[MG];           // chained-operand row of the group
};

template <int KC, int ZT, int CG>
constexpr size_t smem_bytes() {
  // 1024 bytes of alignment slack, the ring, the Z tile, the barriers and the work plan
  using RG = Ring<KC, ZT, CG>;
  return 1024 + RG::NS * RG::STAGEB + RG::ZSMEM + sizeof(Shared<RG::NS>);
}
static_assert(smem_bytes<64, 0, 1>() <= 232448 && smem_bytes<64, 1, 1>() <= 232448 &&
                  smem_bytes<32, 0, 1>() <= 232448 && smem_bytes<32, 1, 1>() <= 232448 &&
                  smem_bytes<64, 2, 1>() <= 232448 && smem_bytes<32, 2, 1>() <= 232448 &&
                  smem_bytes<64, 1, 2>() <= 232448 && smem_bytes<32, 1, 2>() <= 232448 &&
                  smem_bytes<64, 2, 2>() <= 232448 && smem_bytes<32, 2, 2>() <= 232448,
              "every ring geometry fits the 227 KB of shared memory a CTA may use");

// one poll of an mbarrier (acquire at cluster scope when the CTA pair shares it)
template <int CG>
__device__ __forceinline__ bool poll(uint32_t bar, uint32_t parity) {
  return CG == 2 ? mbar_try_cluster(bar, parity) : mbar_try(bar, parity);
}

// bounded wait; one thread polls.  false = the CTA is aborting
template <int CG = 1, class SH>
__device__ __forceinline__ bool wait1(uint32_t bar, uint32_t parity, SH& sh, const TcArgs& a, int code) {
  if (poll<CG>(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (poll<CG>(bar, parity)) return true;
    if (*(volatile int*)&sh.abort_flag) return false;
    if (clock64() - t0 > a.timeout_cycles) {
      *(volatile int*)&sh.abort_flag = 1;
      atomicOr(a.err, code);
      return false;
    }
  }
}

// warp-uniform bounded wait: lane 0 polls, the outcome is broadcast
template <int CG = 1, class SH>
__device__ __forceinline__ bool waitw(uint32_t bar, uint32_t parity, SH& sh, const TcArgs& a, int code) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = wait1<CG>(bar, parity, sh, a, code) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  return ok != 0;
}

// an epilogue warp's arrival on a barrier the MMA thread waits on: the even CTA's copy of it
template <int CG>
__device__ __forceinline__ void arrive_mma_side(uint32_t bar) {
  if (CG == 2) mbar_arrive_cluster(mapa_rank(bar, 0));
  else mbar_arrive(bar);
}

// Failure-path probe: one thread waits, through the passes' own bounded wait, on an mbarrier
// that nothing arrives on; the wait gives up after a.timeout_cycles, sets the error word and
// the kernel returns (the context stays usable)
struct ProbeShared {
  uint64_t bar;
  int abort_flag;
};

__global__ void k_wait_probe(const __grid_constant__ TcArgs a) {
  __shared__ ProbeShared sh;
  if (threadIdx.x == 0) {
    sh.abort_flag = 0;
    mbar_init(smem_u32(&sh.bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    wait1(smem_u32(&sh.bar), 0, sh, a, ERR_TIMEOUT_MMA);
  }
}

// Where a CTA sits in the launch of its pass: block index (x, y, z) and the grid's x extent,
// the launch's own or, in a launch that serves several solves, those of its solve's share.
struct CtaPos {
  int64_t x, nx;
  int y, z;
};

// ---------------- the work plan of a CTA (thread 0): its A tile, chained-operand row and
// groups of B tiles (see the kernel).  CTA pairs (CG = 2) number units of two A tiles.
template <int CG, class SH>
__device__ void plan_work(const TcArgs& a, SH& sh, uint32_t rank, const CtaPos& pos) {
  const int64_t unit = pos.x / CG, nunits = pos.nx / CG;
  int64_t a_row0 = 0;
  int m_y = 0;
  sh.abort_flag = 0;
  int ng = 0;
  if (a.mode == MODE_PASS2) {
    // persistent over work items (row tile rt, column block j), item = rt C + j: CTA c
    // takes items c, c + G, c + 2G, ... (G = the CTAs of the launch), so the CTAs' loads differ by at
    // most one item and neighbouring CTAs share row tiles in L2.  With a block mask the
    // items of the active blocks alone are numbered, in the same order (row block, row
    // tile, active column block), and dealt out the same way.  A CTA pair takes items of
    // two row tiles (its CTAs the first and the second), paired within each row block.
    auto add_item = [&](int64_t arow, int i, int j, bool phantom) {
      sh.g_b0[ng] = a.col_slot[j];
      sh.g_nt[ng] = (int)ceil_div(a.col_size[j], 128);
      sh.g_out[ng] = phantom ? nullptr : a.out + j * a.out_block_stride + arow * a.mpad;
      sh.g_arow[ng] = arow;
      sh.g_my[ng] = i * a.mpad;
      ++ng;
    };
    if (CG == 1 && !a.bmask) {
      const int64_t nitems = a.nrow_tiles * a.C;
      for (int64_t it = pos.x; it < nitems && ng < SH::maxg; it += pos.nx) {
        const int64_t arow = (it / a.C) * 128;
        const int j = (int)(it % a.C);
        int i = 0;
        while (i + 1 < a.R && a.row_slot[i + 1] <= arow) ++i;
        add_item(arow, i, j, false);
      }
    } else {
      int64_t q = unit, first = 0;   // next item of this CTA (pair); first item of row block i
      for (int i = 0; i < a.R && ng < SH::maxg; ++i) {
        int na = 0;
        for (int j = 0; j < a.C; ++j) na += (!a.bmask || a.bmask[i * a.C + j]) ? 1 : 0;
        const int64_t end = (i + 1 < a.R) ? a.row_slot[i + 1] : a.nrow_tiles * 128;
        const int64_t tiles = (end - a.row_slot[i]) / 128, units = ceil_div(tiles, CG);
        const int64_t cnt = units * na;
        for (; q < first + cnt && ng < SH::maxg; q += nunits) {
          const int64_t local = q - first;
          int jj = (int)(local % na), j = 0;
          while ((a.bmask && !a.bmask[i * a.C + j]) || jj-- > 0) ++j;   // the jj-th active column block
          const int64_t tile = (local / na) * CG + rank;
          add_item(a.row_slot[i] + tile * 128, i, j, tile >= tiles);
        }
        first += cnt;
      }
    }
    if (ng > 0) {
      a_row0 = sh.g_arow[0];
      m_y = sh.g_my[0];
    }
  } else if (a.mode == MODE_PREDICT) {
    a_row0 = pos.x * 128;
    m_y = 0;
    {
      // scoring: the features in groups of up to PRED_GT tiles, each group accumulated in
      // a fresh acc2 and added into the output rows in FP32 (the tensor cores' accumulator
      // rounds toward zero at every accumulation; shorter chains keep its bias small)
      const bool phantom = a_row0 >= a.a_rows;
      const int ntiles = (int)(a.fslots / 128);
      const int gt = max(PRED_GT, (int)ceil_div(ntiles, SH::maxg));
      for (int t0 = 0; t0 < ntiles && ng < SH::maxg; t0 += gt) {
        sh.g_b0[ng] = (int64_t)t0 * 128;
        sh.g_nt[ng] = min(gt, ntiles - t0);
        sh.g_out[ng] = phantom ? nullptr : a.out + a_row0 * a.mpad;
        ++ng;
      }
    }
  } else if (a.mode == MODE_PASS1) {
    int j = 0;
    bool phantom = false;
    if (CG == 1) {
      a_row0 = pos.x * 128;
      while (j + 1 < a.C && a.col_slot[j + 1] <= a_row0) ++j;
      phantom = a_row0 - a.col_slot[j] >= a.col_size[j];
    } else {
      // pairs of feature tiles within a column block (both CTAs chain the same V_ij)
      int64_t u = unit;
      int64_t ft = ceil_div(a.col_size[0], 128);
      while (j + 1 < a.C && u >= ceil_div(ft, 2)) {
        u -= ceil_div(ft, 2);
        ++j;
        ft = ceil_div(a.col_size[j], 128);
      }
      const int64_t tile = 2 * u + rank;
      a_row0 = a.col_slot[j] + tile * 128;
      phantom = tile >= ft;
    }
    const int i = pos.y, split = pos.z;
    const int64_t nrt = ceil_div(a.row_size[i], 128);
    const int64_t t0 = split * nrt / a.nsplit, t1 = (split + 1) * nrt / a.nsplit;
    m_y = a.m_shared ? 0 : j * a.mpad;
    const bool active = !a.bmask || a.bmask[i * a.C + j];
    // a pair works whenever its first tile is real; a lone phantom CTA has nothing to do
    if (active && (CG == 2 || !phantom) && t1 > t0) {
      sh.g_b0[0] = a.row_slot[i] + t0 * 128;
      sh.g_nt[0] = (int)(t1 - t0);
      sh.g_out[0] = phantom ? nullptr
                            : a.out + ((int64_t)split * a.R + i) * a.out_block_stride + a_row0 * a.mpad;
      ng = 1;
    }
  } else {  // materialisation window
    a_row0 = a.wz_r0 + pos.x * 128;
    sh.g_b0[0] = a.wz_f0;
    sh.g_nt[0] = (int)ceil_div(a.wz_nf, 128);
    sh.g_out[0] = nullptr;
    ng = 1;
  }
  if (a.mode != MODE_PASS2)
    for (int g = 0; g < ng; ++g) {
      sh.g_arow[g] = a_row0;
      sh.g_my[g] = m_y;
    }
  sh.ngroups = ng;
  sh.a_row0 = a_row0;
  sh.m_y = m_y;
}

template <int KC, int ZT, int CG>
__device__ __forceinline__ void regen_body(const TcArgs& a, const CtaPos& pos) {
  using RG = Ring<KC, ZT, CG>;
  constexpr int NSTAGE = RG::NS;
  constexpr uint32_t STAGE_BYTES = RG::STAGEB, TILE_BYTES = RG::TILEB, BTILE_BYTES = RG::BTILEB;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the operand tiles (the swizzle pattern repeats every 1024 bytes)
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  unsigned char* zbuf = base;
  unsigned char* stages = base + RG::ZSMEM;
  Shared<NSTAGE>& sh = *reinterpret_cast<Shared<NSTAGE>*>(stages + NSTAGE * STAGE_BYTES);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const bool chain = a.mode != MODE_WRITEZ;
  constexpr bool ZTMEM = ZT != 0;            // Z tile in tensor memory
  constexpr bool DB = ZT != 1;               // acc1 double-buffered
  constexpr uint32_t ZH = zh_col(ZT), ZL = ZH + 64, A2 = acc2_col(ZT);
  // CTA pair: rank 0 issues the MMAs
  const uint32_t rank = CG == 2 ? cluster_rank() : 0;

  // ---------------- plan: A tile, chain-operand row, groups of B tiles
  if (threadIdx.x == 0) plan_work<CG>(a, sh, rank, pos);
  __syncthreads();
  const int ngroups = sh.ngroups;
  if (ngroups == 0) return;      // nothing valid in this tile (uniform across the CTA, and the pair)
  const int64_t a_row0 = sh.a_row0;

  const uint32_t bar_full = smem_u32(&sh.full[0]), bar_empty = smem_u32(&sh.empty[0]);
  const uint32_t bar_a1f = smem_u32(&sh.acc1_full[0]), bar_a1e = smem_u32(&sh.acc1_empty[0]);
  const uint32_t bar_zf = smem_u32(&sh.z_full), bar_ze = smem_u32(&sh.z_empty);
  const uint32_t bar_a2f = smem_u32(&sh.acc2_full), bar_a2e = smem_u32(&sh.acc2_empty);
  const uint32_t bar_done = smem_u32(&sh.mma_done);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_a1f + 8 * b, 1);
      mbar_init(bar_a1e + 8 * b, CG * NEPI);
    }
    mbar_init(bar_zf, CG * NEPI);
    mbar_init(bar_ze, 1);
    mbar_init(bar_a2f, 1);
    mbar_init(bar_a2e, CG * NEPI);
    mbar_init(bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc<CG>(smem_u32(&sh.tmem_base), TMEM_COLS);
  fence_before();
  __syncthreads();
  if (CG == 2) cluster_sync_all();   // both CTAs' barriers exist before either signals the other's
  fence_after();
  const uint32_t tmem = sh.tmem_base;
  const int nk = a.nk;
  const int mrows = a.mpad / CG;                          // chain-operand rows this CTA holds
  const uint32_t mbytes = (uint32_t)mrows * RG::ROWB;     // one chain operand chunk (hi or lo)

  if (warp == 0) {
    // ================= TMA producer =================
    if (lane == 0) {
      tma_prefetch_desc(&a.tA_hi);
      tma_prefetch_desc(&a.tB_hi);
      // the even CTA's ring barriers count the copies of both CTAs of a pair
      const uint32_t cfull = CG == 2 ? mapa_rank(bar_full, 0) : bar_full;
      uint32_t it = 0;   // ring uses
      bool ok = true;
      int64_t prev_b = -1;
      int prev_my = 0;
      auto load = [&](uint32_t dst, const CUtensorMap* map, int x, int y, int s) {
        if (CG == 2) tma_load_2d_pair(dst, map, x, y, cfull + 8 * s);
        else tma_load_2d(dst, map, x, y, bar_full + 8 * s);
      };
      auto acquire = [&](uint32_t bytes) -> int {
        const int s = it % NSTAGE;
        const uint32_t use = it / NSTAGE;
        if (use > 0 && !wait1<CG>(bar_empty + 8 * s, (use - 1) & 1, sh, a, ERR_TIMEOUT_PRODUCER)) return -1;
        if (rank == 0) mbar_expect_tx(bar_full + 8 * s, CG * bytes);
        ++it;
        return s;
      };
      auto load_chain = [&](int64_t bslot) -> bool {
        for (int c = 0; c < RG::CHUNKS; ++c) {
          const int s = acquire(2 * mbytes);
          if (s < 0) return false;
          const uint32_t dst = smem_u32(stages + s * STAGE_BYTES);
          const int my = prev_my + (int)rank * mrows;
          load(dst, &a.tM_hi, (int)(bslot + KC * c), my, s);
          load(dst + mbytes, &a.tM_lo, (int)(bslot + KC * c), my, s);
        }
        return true;
      };
      for (int g = 0; g < ngroups && ok; ++g) {
        for (int lt = 0; lt < sh.g_nt[g] && ok; ++lt) {
          const int64_t bslot = sh.g_b0[g] + 128 * (int64_t)lt;
          for (int kc = 0; kc < nk && ok; ++kc) {
            const int s = acquire(STAGE_BYTES);
            if (s < 0) { ok = false; break; }
            const uint32_t dst = smem_u32(stages + s * STAGE_BYTES);
            load(dst, &a.tA_hi, kc * KC, (int)sh.g_arow[g], s);
            load(dst + TILE_BYTES, &a.tA_lo, kc * KC, (int)sh.g_arow[g], s);
            load(dst + 2 * TILE_BYTES, &a.tB_hi, kc * KC, (int)(bslot + rank * RG::BROWS), s);
            load(dst + 2 * TILE_BYTES + BTILE_BYTES, &a.tB_lo, kc * KC, (int)(bslot + rank * RG::BROWS), s);
          }
          if (ok && chain && prev_b >= 0) ok = load_chain(prev_b);
          prev_b = bslot;
          prev_my = sh.g_my[g];
        }
      }
      if (ok && chain && prev_b >= 0) ok = load_chain(prev_b);
      // copies in flight finish before the CTA may exit (bounded); in a pair the even CTA's
      // barriers count both CTAs' copies, and the pair leaves together
      if (rank == 0)
        for (uint32_t u = (it > NSTAGE ? it - NSTAGE : 0); u < it; ++u) {
          const int s = u % NSTAGE;
          if (!poll<CG>(bar_full + 8 * s, (u / NSTAGE) & 1)) {
            const long long t0 = clock64();
            while (!poll<CG>(bar_full + 8 * s, (u / NSTAGE) & 1) && clock64() - t0 < a.timeout_cycles) {
            }
          }
        }
    }
  } else if (warp == 1) {
    // ================= MMA issuer (the even CTA of a pair) =================
    if (lane == 0 && rank == 0) {
      const uint32_t id1 = idesc_f16(128 * CG, 128);      // X.G: scaled FP16 splits
      const uint32_t id2 = idesc_f16(128 * CG, a.mpad);   // chain: scaled FP16 splits of Z and M
      uint32_t it = 0;
      int t = 0;            // B tile index (global)
      bool ok = true;
      // chain of tile tc (global index), group g, first/last flags
      auto do_chain = [&](int tc, int g, bool first, bool last) -> bool {
        if (!wait1<CG>(bar_zf, tc & 1, sh, a, ERR_TIMEOUT_MMA)) return false;
        if (first && g > 0 && !wait1<CG>(bar_a2e, (g - 1) & 1, sh, a, ERR_TIMEOUT_MMA)) return false;
        fence_after();
        const uint32_t zhi = smem_u32(zbuf), zlo = zhi + ZBYTES / 2;
        for (int c = 0; c < RG::CHUNKS; ++c) {
          const int s = it % NSTAGE;
          if (!wait1<CG>(bar_full + 8 * s, (it / NSTAGE) & 1, sh, a, ERR_TIMEOUT_MMA)) return false;
          fence_after();
          const uint32_t mhi = smem_u32(stages + s * STAGE_BYTES), mlo = mhi + mbytes;
#pragma unroll
          for (int kk = 0; kk < RG::KSTEPS; ++kk) {
            const int zk = c * RG::KSTEPS + kk;                 // K step within the 128-wide Z tile
            const uint64_t dmh = smem_desc(mhi + kk * 32, RG::SBO, RG::LAYOUT),
                           dml = smem_desc(mlo + kk * 32, RG::SBO, RG::LAYOUT);
            const uint32_t acc = (first && c == 0 && kk == 0) ? 0u : 1u;
            if (ZTMEM) {
              // A = Z from TMEM: 16 K elements = 8 packed columns per step
              const uint32_t azh = tmem + ZH + 8 * zk, azl = tmem + ZL + 8 * zk;
              mma_ts<CG>(tmem + A2, azh, dmh, id2, acc);
              mma_ts<CG>(tmem + A2, azh, dml, id2, 1u);
              mma_ts<CG>(tmem + A2, azl, dmh, id2, 1u);
            } else {
              const uint32_t zo = (zk / 4) * ZATOM + (zk % 4) * 32;
              const uint64_t dzh = sw128_desc(zhi + zo), dzl = sw128_desc(zlo + zo);
              mma_ss<CG>(tmem + A2, dzh, dmh, id2, acc);
              mma_ss<CG>(tmem + A2, dzh, dml, id2, 1u);
              mma_ss<CG>(tmem + A2, dzl, dmh, id2, 1u);
            }
          }
          commit_both<CG>(bar_empty + 8 * s);
          ++it;
        }
        commit_both<CG>(bar_ze);
        if (last) commit_both<CG>(bar_a2f);
        return true;
      };
      int pg = -1, pt = -1;
      bool pfirst = false, plast = false;
      for (int g = 0; g < ngroups && ok; ++g) {
        const int ntg = sh.g_nt[g];
        for (int lt = 0; lt < ntg && ok; ++lt, ++t) {
          // acc1: double-buffered (ZT = 0, 2) or one buffer (ZT = 1)
          const int b = DB ? (t & 1) : 0;
          const bool reuse = DB ? (t >= 2) : (t >= 1);
          const uint32_t par = DB ? (((t - 2) >> 1) & 1) : ((t - 1) & 1);
          if (reuse && !wait1<CG>(bar_a1e + 8 * b, par, sh, a, ERR_TIMEOUT_MMA)) { ok = false; break; }
          fence_after();
          const uint32_t d1 = tmem + 128 * b;
          for (int kc = 0; kc < nk; ++kc) {
            const int s = it % NSTAGE;
            if (!wait1<CG>(bar_full + 8 * s, (it / NSTAGE) & 1, sh, a, ERR_TIMEOUT_MMA)) { ok = false; break; }
            fence_after();
            const uint32_t sa = smem_u32(stages + s * STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < RG::KSTEPS; ++kk) {
              const uint64_t ah = smem_desc(sa + kk * 32, RG::SBO, RG::LAYOUT),
                             al = smem_desc(sa + TILE_BYTES + kk * 32, RG::SBO, RG::LAYOUT);
              const uint64_t bh = smem_desc(sa + 2 * TILE_BYTES + kk * 32, RG::SBO, RG::LAYOUT),
                             bl = smem_desc(sa + 2 * TILE_BYTES + BTILE_BYTES + kk * 32, RG::SBO, RG::LAYOUT);
              mma_ss<CG>(d1, ah, bh, id1, (kc > 0 || kk > 0) ? 1u : 0u);
              mma_ss<CG>(d1, ah, bl, id1, 1u);
              mma_ss<CG>(d1, al, bh, id1, 1u);
            }
            commit_both<CG>(bar_empty + 8 * s);
            ++it;
          }
          if (!ok) break;
          commit_both<CG>(bar_a1f + 8 * b);
          if (chain && pt >= 0) ok = do_chain(pt, pg, pfirst, plast);
          pt = t;
          pg = g;
          pfirst = lt == 0;
          plast = lt == ntg - 1;
        }
      }
      if (ok && chain && pt >= 0) ok = do_chain(pt, pg, pfirst, plast);
      // all products issued by this thread complete before TMEM is released
      commit_own<CG>(bar_done);
      wait1<CG>(bar_done, 0, sh, a, ERR_TIMEOUT_MMA);
    }
  } else {
    // ================= epilogue =================
    const int ew = warp - 2;                 // 0..7
    const int quarter = warp & 3;            // TMEM lane quarter of this warp
    const int colbase = (ew < 4) ? 0 : 64;   // accumulator columns of this warp
    const int row = quarter * 32 + lane;     // row of the A tile (TMEM lane)
    const int64_t arow = a_row0 + row;
    // No masks: padding rows and features meet zero chain operands (V and W' are
    // zero there), and materialisation writes only the valid window.  The phase b
    // is either part of the product (column of ones in X) or added here.
    const bool add_bias = !a.bias_in_mma;
    const float inv_xg = a.inv_xg;            // power of two: the rescaling is exact
    // (a discarded feature tile of a CTA pair may lie past the last feature slot)
    const float bias_a =
        (add_bias && a.mode == MODE_PASS1 && arow < a.fslots && RFF_IN(arow, a.fslots)) ? a.bias[arow] : 0.f;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    int t = 0;
    bool ok = true;
    for (int g = 0; g < ngroups && ok; ++g) {
      const int ntg = sh.g_nt[g];
      for (int lt = 0; lt < ntg && ok; ++lt, ++t) {
        const int b = DB ? (t & 1) : 0;
        const int64_t bslot = sh.g_b0[g] + 128 * (int64_t)lt;
        if (!waitw<CG>(bar_a1f + 8 * b, DB ? ((t >> 1) & 1) : (t & 1), sh, a, ERR_TIMEOUT_EPI)) { ok = false; break; }
        fence_after();
        uint32_t v0[32], v1[32];
        tmem_ld32(tmem + lane_addr + 128 * b + colbase, v0);
        tmem_ld32(tmem + lane_addr + 128 * b + colbase + 32, v1);
        tmem_wait_ld();
        fence_before();
        __syncwarp();
        if (lane == 0) arrive_mma_side<CG>(bar_a1e + 8 * b);
        // z = cos(acc (+ b)), times COS_SCALE when it feeds the chained product; the factor
        // sqrt(2/D) is applied when acc2 (or the materialised Z) is written
        float z[64];
        if (add_bias) {
          const float* bcol = a.bias + bslot + colbase;
#pragma unroll
          for (int c = 0; c < 64; ++c) {
            const float ph = (a.mode == MODE_PASS1)                             ? bias_a
                             : RFF_IN(bslot + colbase + c, a.fslots) ? __ldg(bcol + c)
                                                                     : 0.f;
            z[c] = __uint_as_float(c < 32 ? v0[c] : v1[c - 32]) * inv_xg + ph;
          }
          // one loop per branch: a per-element choice would evaluate both cosines
          if (chain) {
#pragma unroll
            for (int c = 0; c < 64; ++c) z[c] = cos_rr_pow2<7>(z[c]);
          } else {
#pragma unroll
            for (int c = 0; c < 64; ++c) z[c] = cos_rr(z[c]);
          }
        } else {
#pragma unroll
          for (int c = 0; c < 64; ++c) z[c] = __uint_as_float(c < 32 ? v0[c] : v1[c - 32]) * inv_xg;
          if (chain) {
#pragma unroll
            for (int c = 0; c < 64; ++c) z[c] = cos_rr_pow2<7>(z[c]);
          } else {
#pragma unroll
            for (int c = 0; c < 64; ++c) z[c] = cos_rr(z[c]);
          }
        }
        if (!chain) {
          // materialise Z = sqrt(2/D) cos(...) (float32) inside the window
          const int64_t r = arow - a.wz_r0;
          if (r < a.wz_nr && a.zt_hi) {
            // transposed FP16 hi/lo split of zt_scale Z: the lanes hold consecutive rows, so
            // every store of the warp fills 32 consecutive elements of one row of Z^T
#pragma unroll
            for (int c = 0; c < 64; ++c) {
              const int64_t f = bslot + colbase + c - a.wz_f0;
              if (f < a.wz_nf && RFF_IN(f * a.ldo + r, a.out_elems)) {
                const float xs = a.scale * z[c] * a.zt_scale;
                const __half h = __float2half_rn(xs);
                a.zt_hi[f * a.ldo + r] = h;
                a.zt_lo[f * a.ldo + r] = __float2half_rn(xs - __half2float(h));
              }
            }
          } else if (r < a.wz_nr) {
#pragma unroll
            for (int c = 0; c < 64; ++c) {
              const int64_t f = bslot + colbase + c - a.wz_f0;
              if (f < a.wz_nf && RFF_IN(r * a.ldo + f, a.out_elems)) a.out[r * a.ldo + f] = a.scale * z[c];
            }
          }
          continue;
        }
        // Z tile must be free: the chain of the previous tile has completed
        if (t >= 1 && !waitw<CG>(bar_ze, (t - 1) & 1, sh, a, ERR_TIMEOUT_EPI)) { ok = false; break; }
        if (ZTMEM) {
          // split COS_SCALE z into hi/lo FP16 pairs (two K elements per 32-bit column) and
          // store this warp's 32 rows x 64 features into the Z columns of TMEM
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
            uint32_t ph[16], pl[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const float z0 = z[32 * hf + 2 * q], z1 = z[32 * hf + 2 * q + 1];   // COS_SCALE z
              const __half2 h = __floats2half2_rn(z0, z1);
              const float2 f = __half22float2(h);
              const __half2 l = __floats2half2_rn(z0 - f.x, z1 - f.y);
              ph[q] = *reinterpret_cast<const uint32_t*>(&h);
              pl[q] = *reinterpret_cast<const uint32_t*>(&l);
            }
            const uint32_t col = (uint32_t)(colbase / 2 + 16 * hf);
            tmem_st16(tmem + lane_addr + ZH + col, ph);
            tmem_st16(tmem + lane_addr + ZL + col, pl);
          }
          tmem_wait_st();
          fence_before();
        } else {
          // split into hi/lo FP16 and store in the 128-byte swizzled K-major layout
          unsigned char* zhi = zbuf + (colbase / 64) * ZATOM;
          unsigned char* zlo = zhi + ZBYTES / 2;
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            uint32_t ph[4], pl[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              // hi = fp16x2(s z0, s z1); lo = fp16x2(s z - hi) (packed conversions)
              const float z0 = z[ch * 8 + 2 * q], z1 = z[ch * 8 + 2 * q + 1];   // COS_SCALE z
              const __half2 h = __floats2half2_rn(z0, z1);
              const float2 hf = __half22float2(h);
              const __half2 l = __floats2half2_rn(z0 - hf.x, z1 - hf.y);
              ph[q] = *reinterpret_cast<const uint32_t*>(&h);
              pl[q] = *reinterpret_cast<const uint32_t*>(&l);
            }
            const uint32_t off = row * 128 + ((ch ^ (row & 7)) << 4);
            *reinterpret_cast<uint4*>(zhi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
            *reinterpret_cast<uint4*>(zlo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
          }
          fence_proxy_async();
        }
        __syncwarp();
        if (lane == 0) arrive_mma_side<CG>(bar_zf);
        if (lt == ntg - 1) {
          // group finished: write acc2 (rows of this warp, half of the m_pad columns)
          if (!waitw<CG>(bar_a2f, g & 1, sh, a, ERR_TIMEOUT_EPI)) { ok = false; break; }
          fence_after();
          if (sh.g_out[g]) {   // a discarded tile of a CTA pair writes nothing
            const int half = a.mpad / 2;
            const int c0 = (ew < 4) ? 0 : half;
            float* orow = sh.g_out[g] + (int64_t)row * a.mpad;
            // undo the FP16 scales of Z (COS_SCALE) and of the chained operand, apply sqrt(2/D)
            const float sc = a.scale / COS_SCALE * (a.m_amax ? f16_inv_scale(__uint_as_float(*a.m_amax)) : 1.f);
            float omx = 0.f;
            for (int c = 0; c < half; c += 8) {
              uint32_t r8[8];
              tmem_ld8(tmem + lane_addr + A2 + c0 + c, r8);
              tmem_wait_ld();
              float4* dst = reinterpret_cast<float4*>(orow + c0 + c);
              float4 v0 = make_float4(sc * __uint_as_float(r8[0]), sc * __uint_as_float(r8[1]),
                                      sc * __uint_as_float(r8[2]), sc * __uint_as_float(r8[3]));
              float4 v1 = make_float4(sc * __uint_as_float(r8[4]), sc * __uint_as_float(r8[5]),
                                      sc * __uint_as_float(r8[6]), sc * __uint_as_float(r8[7]));
              const bool in = RFF_SPAN(orow + c0 + c - a.out, 8, a.out_elems);
              if (in && a.mode == MODE_PREDICT && g > 0) {   // this CTA wrote these rows for group g-1
                const float4 p0 = dst[0], p1 = dst[1];
                v0 = make_float4(p0.x + v0.x, p0.y + v0.y, p0.z + v0.z, p0.w + v0.w);
                v1 = make_float4(p1.x + v1.x, p1.y + v1.y, p1.z + v1.z, p1.w + v1.w);
              }
              if (in) {
                dst[0] = v0;
                dst[1] = v1;
              }
              omx = fmaxf(omx, fmaxf(fmaxf(fmaxf(fabsf(v0.x), fabsf(v0.y)), fmaxf(fabsf(v0.z), fabsf(v0.w))),
                                     fmaxf(fmaxf(fabsf(v1.x), fabsf(v1.y)), fmaxf(fabsf(v1.z), fabsf(v1.w)))));
            }
            if (a.out_amax) {
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) omx = fmaxf(omx, __shfl_xor_sync(0xffffffffu, omx, o));
              if (lane == 0 && omx > 0.f) atomicMax(a.out_amax, __float_as_uint(omx));
            }
          }
          fence_before();
          __syncwarp();
          if (lane == 0) arrive_mma_side<CG>(bar_a2e);
        }
      }
    }
  }
  // ---------------- teardown
  fence_before();
  __syncthreads();
  if (CG == 2) cluster_sync_all();   // neither CTA of a pair leaves while the other may still use it
  fence_after();
  if (warp == 1) tmem_dealloc<CG>(tmem, TMEM_COLS);
}

template <int KC, int ZT, int CG>
__global__ void __launch_bounds__(NTHREADS, 1) k_regen_tc(const __grid_constant__ TcArgs a) {
  regen_body<KC, ZT, CG>(a, CtaPos{(int64_t)blockIdx.x, (int64_t)gridDim.x, (int)blockIdx.y, (int)blockIdx.z});
}

// One launch for the same pass of several solves (a model-selection sweep): solve g owns the
// CTAs [start[g], start[g+1]) of the one-dimensional grid, laid out as its own launch would
// be (gx[g] x gy[g] x gz[g], x fastest), and its arguments, tensor maps included, are entry g
// of a table in device memory.  The solves' CTAs run side by side in one grid, so the SMs a
// small solve leaves free take CTAs of the others instead of idling until another launch.
constexpr int MULTI_MAX = 64;
struct MultiArgs {
  const TcArgs* table;   // device, ngroups entries (64-byte aligned: the tensor maps)
  int ngroups;
  int64_t start[MULTI_MAX + 1];
  int64_t gx[MULTI_MAX];
  int gy[MULTI_MAX];
};

template <int KC, int ZT>
__global__ void __launch_bounds__(NTHREADS, 1) k_regen_multi(const __grid_constant__ MultiArgs m) {
  const int64_t b = blockIdx.x;
  int g = 0;
  while (g + 1 < m.ngroups && b >= m.start[g + 1]) ++g;
  const int64_t local = b - m.start[g];
  const int64_t gx = m.gx[g];
  const int64_t yz = local / gx;
  regen_body<KC, ZT, 1>(m.table[g], CtaPos{local % gx, gx, (int)(yz % m.gy[g]), (int)(yz / m.gy[g])});
}

// ------------------------------------------------------------------ the wide geometry
// X.G with N = 256: every MMA multiplies the CTA's 128-row A tile by 256 B rows (two
// 128-row B tiles), so a K step's three products read 4 + 8 KB of shared memory per 128
// tensor-pipe cycles (96 B per cycle) instead of 4 + 4 KB per 64 (128 B per cycle, the
// whole shared-memory bandwidth, so that every byte the TMA ring writes stalls the tensor
// pipe), and the ring writes 96 KB per 1,536 product cycles instead of 64 KB per 768.
// acc1 takes 256 TMEM columns; the Z tile of each 128-feature half goes to TMEM (hi, 64
// columns) and shared memory (lo, 32 KB, the chained MMA reads it by descriptor), and acc2
// follows at column 320 (m_pad <= 192).  The two halves of a B pair are chained one after
// the other through the one Z tile; a half past the end of its group (an odd tile count) is
// computed and not chained.  Products and their order per output element are those of the
// other geometries: results are bit-identical.
constexpr uint32_t W_ZH = 256, W_A2 = 320;
constexpr int W_MAX_MPAD = 192;
constexpr int W_MAXG = 48;   // fewer groups per CTA than MAXG: the plan's arrays must fit beside the ring

template <int KC>
struct WideRing {
  static constexpr uint32_t ROWB = KC * 2;
  static constexpr uint32_t TILEB = 128 * ROWB;            // A hi or lo
  static constexpr uint32_t BTILEB = 256 * ROWB;           // B hi or lo: a pair of B tiles
  static constexpr uint32_t STAGEB = 2 * TILEB + 2 * BTILEB;
  static constexpr int NS = (KC == 64) ? 2 : 4;
  static constexpr int KSTEPS = KC / 16;
  static constexpr int CHUNKS = 128 / KC;                  // chain-operand chunks per 128-feature half
  static constexpr uint32_t LAYOUT = (KC == 64) ? 2 : 4;
  static constexpr uint32_t SBO = 8 * ROWB;
  static constexpr uint32_t ZLO = ZBYTES / 2;              // Z lo: 128 x 128 FP16, two 64-column atoms
};
template <int KC>
constexpr size_t wide_smem_bytes() {
  using RG = WideRing<KC>;
  return 1024 + RG::ZLO + RG::NS * RG::STAGEB + sizeof(Shared<RG::NS, W_MAXG>);
}
static_assert(wide_smem_bytes<64>() <= 232448 && wide_smem_bytes<32>() <= 232448,
              "the wide ring and the Z lo tile fit the 227 KB of shared memory a CTA may use");

template <int KC>
__global__ void __launch_bounds__(NTHREADS, 1) k_regen_wide(const __grid_constant__ TcArgs a) {
  using RG = WideRing<KC>;
  constexpr int NSTAGE = RG::NS;
  constexpr uint32_t STAGE_BYTES = RG::STAGEB, TILE_BYTES = RG::TILEB, BTILE_BYTES = RG::BTILEB;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  unsigned char* zlo_buf = base;                            // Z lo, 128-byte swizzled K-major
  unsigned char* stages = base + RG::ZLO;
  Shared<NSTAGE, W_MAXG>& sh = *reinterpret_cast<Shared<NSTAGE, W_MAXG>*>(stages + NSTAGE * STAGE_BYTES);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const bool chain = a.mode != MODE_WRITEZ;

  if (threadIdx.x == 0)
    plan_work<1>(a, sh, 0, CtaPos{(int64_t)blockIdx.x, (int64_t)gridDim.x, (int)blockIdx.y, (int)blockIdx.z});
  __syncthreads();
  const int ngroups = sh.ngroups;
  if (ngroups == 0) return;
  const int64_t a_row0 = sh.a_row0;

  const uint32_t bar_full = smem_u32(&sh.full[0]), bar_empty = smem_u32(&sh.empty[0]);
  const uint32_t bar_a1f = smem_u32(&sh.acc1_full[0]), bar_a1e = smem_u32(&sh.acc1_empty[0]);
  const uint32_t bar_zf = smem_u32(&sh.z_full), bar_ze = smem_u32(&sh.z_empty);
  const uint32_t bar_a2f = smem_u32(&sh.acc2_full), bar_a2e = smem_u32(&sh.acc2_empty);
  const uint32_t bar_done = smem_u32(&sh.mma_done);
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_a1f, 1);
    mbar_init(bar_a1e, NEPI);
    mbar_init(bar_zf, NEPI);
    mbar_init(bar_ze, 1);
    mbar_init(bar_a2f, 1);
    mbar_init(bar_a2e, NEPI);
    mbar_init(bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc<1>(smem_u32(&sh.tmem_base), TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sh.tmem_base;
  const int nk = a.nk;
  const uint32_t mbytes = (uint32_t)a.mpad * RG::ROWB;    // one chain operand chunk (hi or lo)

  if (warp == 0) {
    // ================= TMA producer =================
    if (lane == 0) {
      tma_prefetch_desc(&a.tA_hi);
      tma_prefetch_desc(&a.tB_hi);
      uint32_t it = 0;
      bool ok = true;
      int64_t prev_b = -1;
      int prev_my = 0, prev_halves = 0;
      auto acquire = [&](uint32_t bytes) -> int {
        const int s = it % NSTAGE;
        const uint32_t use = it / NSTAGE;
        if (use > 0 && !wait1(bar_empty + 8 * s, (use - 1) & 1, sh, a, ERR_TIMEOUT_PRODUCER)) return -1;
        mbar_expect_tx(bar_full + 8 * s, bytes);
        ++it;
        return s;
      };
      auto load_chain = [&]() -> bool {
        for (int h = 0; h < prev_halves; ++h)
          for (int c = 0; c < RG::CHUNKS; ++c) {
            const int s = acquire(2 * mbytes);
            if (s < 0) return false;
            const uint32_t dst = smem_u32(stages + s * STAGE_BYTES);
            const int x = (int)(prev_b + 128 * h + KC * c);
            tma_load_2d(dst, &a.tM_hi, x, prev_my, bar_full + 8 * s);
            tma_load_2d(dst + mbytes, &a.tM_lo, x, prev_my, bar_full + 8 * s);
          }
        return true;
      };
      for (int g = 0; g < ngroups && ok; ++g) {
        const int ntg = sh.g_nt[g];
        for (int lt = 0; lt < ntg && ok; lt += 2) {
          const int64_t bslot = sh.g_b0[g] + 128 * (int64_t)lt;
          for (int kc = 0; kc < nk && ok; ++kc) {
            const int s = acquire(STAGE_BYTES);
            if (s < 0) { ok = false; break; }
            const uint32_t dst = smem_u32(stages + s * STAGE_BYTES);
            const uint32_t fb = bar_full + 8 * s;
            tma_load_2d(dst, &a.tA_hi, kc * KC, (int)sh.g_arow[g], fb);
            tma_load_2d(dst + TILE_BYTES, &a.tA_lo, kc * KC, (int)sh.g_arow[g], fb);
            tma_load_2d(dst + 2 * TILE_BYTES, &a.tB_hi, kc * KC, (int)bslot, fb);
            tma_load_2d(dst + 2 * TILE_BYTES + BTILE_BYTES, &a.tB_lo, kc * KC, (int)bslot, fb);
          }
          if (ok && chain && prev_b >= 0) ok = load_chain();
          prev_b = bslot;
          prev_my = sh.g_my[g];
          prev_halves = (lt + 1 < ntg) ? 2 : 1;
        }
      }
      if (ok && chain && prev_b >= 0) ok = load_chain();
      for (uint32_t u = (it > NSTAGE ? it - NSTAGE : 0); u < it; ++u) {
        const int s = u % NSTAGE;
        if (!mbar_try(bar_full + 8 * s, (u / NSTAGE) & 1)) {
          const long long t0 = clock64();
          while (!mbar_try(bar_full + 8 * s, (u / NSTAGE) & 1) && clock64() - t0 < a.timeout_cycles) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer =================
    if (lane == 0) {
      const uint32_t id1 = idesc_f16(128, 256);
      const uint32_t id2 = idesc_f16(128, a.mpad);
      uint32_t it = 0, zu = 0;   // ring uses; Z tile uses
      int t = 0;                 // B pair index (global)
      bool ok = true;
      // the chains of B pair (group g, first pair of the group?, last pair?, halves)
      auto do_chain = [&](int g, bool first, bool last, int halves) -> bool {
        for (int h = 0; h < halves; ++h, ++zu) {
          if (!wait1(bar_zf, zu & 1, sh, a, ERR_TIMEOUT_MMA)) return false;
          const bool fresh = first && h == 0;
          if (fresh && g > 0 && !wait1(bar_a2e, (g - 1) & 1, sh, a, ERR_TIMEOUT_MMA)) return false;
          fence_after();
          const uint32_t zlo = smem_u32(zlo_buf);
          for (int c = 0; c < RG::CHUNKS; ++c) {
            const int s = it % NSTAGE;
            if (!wait1(bar_full + 8 * s, (it / NSTAGE) & 1, sh, a, ERR_TIMEOUT_MMA)) return false;
            fence_after();
            const uint32_t mhi = smem_u32(stages + s * STAGE_BYTES), mlo = mhi + mbytes;
#pragma unroll
            for (int kk = 0; kk < RG::KSTEPS; ++kk) {
              const int zk = c * RG::KSTEPS + kk;
              const uint64_t dmh = smem_desc(mhi + kk * 32, RG::SBO, RG::LAYOUT),
                             dml = smem_desc(mlo + kk * 32, RG::SBO, RG::LAYOUT);
              const uint32_t acc = (fresh && c == 0 && kk == 0) ? 0u : 1u;
              const uint32_t azh = tmem + W_ZH + 8 * zk;
              const uint32_t zo = (zk / 4) * ZATOM + (zk % 4) * 32;
              mma_bf16_ts(tmem + W_A2, azh, dmh, id2, acc);
              mma_bf16_ts(tmem + W_A2, azh, dml, id2, 1u);
              mma_bf16(tmem + W_A2, sw128_desc(zlo + zo), dmh, id2, 1u);
            }
            mma_commit(bar_empty + 8 * s);
            ++it;
          }
          mma_commit(bar_ze);
          if (last && h == halves - 1) mma_commit(bar_a2f);
        }
        return true;
      };
      int pg = -1, phalves = 0;
      bool pfirst = false, plast = false;
      for (int g = 0; g < ngroups && ok; ++g) {
        const int ntg = sh.g_nt[g];
        for (int lt = 0; lt < ntg && ok; lt += 2, ++t) {
          if (t >= 1 && !wait1(bar_a1e, (t - 1) & 1, sh, a, ERR_TIMEOUT_MMA)) { ok = false; break; }
          fence_after();
          for (int kc = 0; kc < nk; ++kc) {
            const int s = it % NSTAGE;
            if (!wait1(bar_full + 8 * s, (it / NSTAGE) & 1, sh, a, ERR_TIMEOUT_MMA)) { ok = false; break; }
            fence_after();
            const uint32_t sa = smem_u32(stages + s * STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < RG::KSTEPS; ++kk) {
              const uint64_t ah = smem_desc(sa + kk * 32, RG::SBO, RG::LAYOUT),
                             al = smem_desc(sa + TILE_BYTES + kk * 32, RG::SBO, RG::LAYOUT);
              const uint64_t bh = smem_desc(sa + 2 * TILE_BYTES + kk * 32, RG::SBO, RG::LAYOUT),
                             bl = smem_desc(sa + 2 * TILE_BYTES + BTILE_BYTES + kk * 32, RG::SBO, RG::LAYOUT);
              mma_bf16(tmem, ah, bh, id1, (kc > 0 || kk > 0) ? 1u : 0u);
              mma_bf16(tmem, ah, bl, id1, 1u);
              mma_bf16(tmem, al, bh, id1, 1u);
            }
            mma_commit(bar_empty + 8 * s);
            ++it;
          }
          if (!ok) break;
          mma_commit(bar_a1f);
          if (chain && pg >= 0) ok = do_chain(pg, pfirst, plast, phalves);
          pg = g;
          pfirst = lt == 0;
          plast = lt + 2 >= ntg;
          phalves = (lt + 1 < ntg) ? 2 : 1;
        }
      }
      if (ok && chain && pg >= 0) ok = do_chain(pg, pfirst, plast, phalves);
      mma_commit(bar_done);
      wait1(bar_done, 0, sh, a, ERR_TIMEOUT_MMA);
    }
  } else {
    // ================= epilogue =================
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int colbase = (ew < 4) ? 0 : 64;
    const int row = quarter * 32 + lane;
    const int64_t arow = a_row0 + row;
    const bool add_bias = !a.bias_in_mma;
    const float inv_xg = a.inv_xg;
    const float bias_a =
        (add_bias && a.mode == MODE_PASS1 && arow < a.fslots && RFF_IN(arow, a.fslots)) ? a.bias[arow] : 0.f;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    int t = 0;
    uint32_t zu = 0;
    bool ok = true;
    for (int g = 0; g < ngroups && ok; ++g) {
      const int ntg = sh.g_nt[g];
      for (int lt = 0; lt < ntg && ok; lt += 2, ++t) {
        if (!waitw(bar_a1f, t & 1, sh, a, ERR_TIMEOUT_EPI)) { ok = false; break; }
        fence_after();
        const int halves = (lt + 1 < ntg) ? 2 : 1;
        for (int h = 0; h < 2 && ok; ++h) {
          const int64_t bslot = sh.g_b0[g] + 128 * (int64_t)(lt + h);
          uint32_t v0[32], v1[32];
          tmem_ld32(tmem + lane_addr + 128 * h + colbase, v0);
          tmem_ld32(tmem + lane_addr + 128 * h + colbase + 32, v1);
          tmem_wait_ld();
          if (h == 1) {   // both halves read out: the next X.G may overwrite acc1
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_a1e);
          }
          if (h >= halves && chain) continue;    // a half past the group: computed, not chained
          float z[64];
          if (add_bias) {
            const float* bcol = a.bias + bslot + colbase;
#pragma unroll
            for (int c = 0; c < 64; ++c) {
              const float ph = (a.mode == MODE_PASS1)                             ? bias_a
                               : RFF_IN(bslot + colbase + c, a.fslots) ? __ldg(bcol + c)
                                                                       : 0.f;
              z[c] = __uint_as_float(c < 32 ? v0[c] : v1[c - 32]) * inv_xg + ph;
            }
          } else {
#pragma unroll
            for (int c = 0; c < 64; ++c) z[c] = __uint_as_float(c < 32 ? v0[c] : v1[c - 32]) * inv_xg;
          }
          // one loop per branch: a per-element choice would evaluate both cosines
          if (chain) {
#pragma unroll
            for (int c = 0; c < 64; ++c) z[c] = cos_rr_pow2<7>(z[c]);
          } else {
#pragma unroll
            for (int c = 0; c < 64; ++c) z[c] = cos_rr(z[c]);
          }
          if (!chain) {
            const int64_t r = arow - a.wz_r0;
            if (r < a.wz_nr && a.zt_hi) {
#pragma unroll
              for (int c = 0; c < 64; ++c) {
                const int64_t f = bslot + colbase + c - a.wz_f0;
                if (f >= 0 && f < a.wz_nf && RFF_IN(f * a.ldo + r, a.out_elems)) {
                  const float xs = a.scale * z[c] * a.zt_scale;
                  const __half hh = __float2half_rn(xs);
                  a.zt_hi[f * a.ldo + r] = hh;
                  a.zt_lo[f * a.ldo + r] = __float2half_rn(xs - __half2float(hh));
                }
              }
            } else if (r < a.wz_nr) {
#pragma unroll
              for (int c = 0; c < 64; ++c) {
                const int64_t f = bslot + colbase + c - a.wz_f0;
                if (f >= 0 && f < a.wz_nf && RFF_IN(r * a.ldo + f, a.out_elems)) a.out[r * a.ldo + f] = a.scale * z[c];
              }
            }
            continue;
          }
          // the Z tile is free once the previous half's chain has completed
          if (zu >= 1 && !waitw(bar_ze, (zu - 1) & 1, sh, a, ERR_TIMEOUT_EPI)) { ok = false; break; }
          {
            // hi: FP16 pairs into the Z columns of TMEM; lo: the swizzled K-major tile in shared memory
            unsigned char* zl = zlo_buf + (colbase / 64) * ZATOM;
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
              uint32_t ph[16], pl[16];
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const float z0 = z[32 * hf + 2 * q], z1 = z[32 * hf + 2 * q + 1];   // COS_SCALE z
                const __half2 hh = __floats2half2_rn(z0, z1);
                const float2 f = __half22float2(hh);
                const __half2 l = __floats2half2_rn(z0 - f.x, z1 - f.y);
                ph[q] = *reinterpret_cast<const uint32_t*>(&hh);
                pl[q] = *reinterpret_cast<const uint32_t*>(&l);
              }
              tmem_st16(tmem + lane_addr + W_ZH + (uint32_t)(colbase / 2 + 16 * hf), ph);
              // 16 packed words = 32 features = four 16-byte chunks of this row
#pragma unroll
              for (int q4 = 0; q4 < 4; ++q4) {
                const int ch = 4 * hf + q4;
                const uint32_t off = row * 128 + ((ch ^ (row & 7)) << 4);
                *reinterpret_cast<uint4*>(zl + off) = make_uint4(pl[4 * q4], pl[4 * q4 + 1], pl[4 * q4 + 2], pl[4 * q4 + 3]);
              }
            }
            tmem_wait_st();
            fence_proxy_async();
            fence_before();
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(bar_zf);
          ++zu;
        }
        if (!ok) break;
        if (chain && lt + 2 >= ntg) {
          if (!waitw(bar_a2f, g & 1, sh, a, ERR_TIMEOUT_EPI)) { ok = false; break; }
          fence_after();
          if (sh.g_out[g]) {
            const int half = a.mpad / 2;
            const int c0 = (ew < 4) ? 0 : half;
            float* orow = sh.g_out[g] + (int64_t)row * a.mpad;
            const float sc = a.scale / COS_SCALE * (a.m_amax ? f16_inv_scale(__uint_as_float(*a.m_amax)) : 1.f);
            float omx = 0.f;
            for (int c = 0; c < half; c += 8) {
              uint32_t r8[8];
              tmem_ld8(tmem + lane_addr + W_A2 + c0 + c, r8);
              tmem_wait_ld();
              float4* dst = reinterpret_cast<float4*>(orow + c0 + c);
              float4 v0 = make_float4(sc * __uint_as_float(r8[0]), sc * __uint_as_float(r8[1]),
                                      sc * __uint_as_float(r8[2]), sc * __uint_as_float(r8[3]));
              float4 v1 = make_float4(sc * __uint_as_float(r8[4]), sc * __uint_as_float(r8[5]),
                                      sc * __uint_as_float(r8[6]), sc * __uint_as_float(r8[7]));
              const bool in = RFF_SPAN(orow + c0 + c - a.out, 8, a.out_elems);
              if (in && a.mode == MODE_PREDICT && g > 0) {
                const float4 p0 = dst[0], p1 = dst[1];
                v0 = make_float4(p0.x + v0.x, p0.y + v0.y, p0.z + v0.z, p0.w + v0.w);
                v1 = make_float4(p1.x + v1.x, p1.y + v1.y, p1.z + v1.z, p1.w + v1.w);
              }
              if (in) {
                dst[0] = v0;
                dst[1] = v1;
              }
              omx = fmaxf(omx, fmaxf(fmaxf(fmaxf(fabsf(v0.x), fabsf(v0.y)), fmaxf(fabsf(v0.z), fabsf(v0.w))),
                                     fmaxf(fmaxf(fabsf(v1.x), fabsf(v1.y)), fmaxf(fabsf(v1.z), fabsf(v1.w)))));
            }
            if (a.out_amax) {
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) omx = fmaxf(omx, __shfl_xor_sync(0xffffffffu, omx, o));
              if (lane == 0 && omx > 0.f) atomicMax(a.out_amax, __float_as_uint(omx));
            }
          }
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar_a2e);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc<1>(tmem, TMEM_COLS);
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// K chunk of the ring (64: 128-byte swizzle, 2 or 3 stages; 32: 64-byte swizzle, 4 or 6 stages).
// Measured on the multiclass workload: 64 is ~5 % faster (both are bound by shared-
// memory bandwidth, see the profile notes), so it is the default; RFF_TC_KCHUNK=32
// in the environment selects the other ring.
int ring_kc() {
  static int kc = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* e = getenv("RFF_TC_KCHUNK");
    kc = (e && atoi(e) == 32) ? 32 : 64;
  });
  return kc;
}

// 2-D BF16 tensor [rows][cols] (cols contiguous, leading dimension ld elements),
// box of kc columns x box_rows rows, swizzled to match the ring layout
cudaError_t make_map(CUtensorMap* m, const void* ptr, int64_t cols, int64_t rows, int64_t ld, int box_rows,
                     int kc) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (ld * 2) % 16 || box_rows > 256 || box_rows < 1)
    return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)kc, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, kc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int KC, int ZT, int CG>
cudaError_t launch_geom(TcArgs& a, dim3 grid, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_regen_tc<KC, ZT, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_bytes<KC, ZT, CG>());
  });
  if (attr_err != cudaSuccess) return attr_err;
  if (CG == 1) {
    k_regen_tc<KC, ZT, CG><<<grid, NTHREADS, smem_bytes<KC, ZT, CG>(), st>>>(a);
    return cudaGetLastError();
  }
  // CTA pairs: clusters of two along x (the grid's x extent is even)
  if (grid.x % 2) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = smem_bytes<KC, ZT, CG>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_regen_tc<KC, ZT, CG>, a);
}

template <int KC>
cudaError_t launch_wide(TcArgs& a, dim3 grid, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_regen_wide<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)wide_smem_bytes<KC>());
  });
  if (attr_err != cudaSuccess) return attr_err;
  k_regen_wide<KC><<<grid, NTHREADS, wide_smem_bytes<KC>(), st>>>(a);
  return cudaGetLastError();
}

// zt 3: the wide geometry (N = 256 X.G products; one CTA)
cudaError_t launch(TcArgs& a, dim3 grid, cudaStream_t st, int kc, int zt, int cg) {
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
  if (zt == 3) {
    if (a.mpad > W_MAX_MPAD) return cudaErrorInvalidValue;   // acc1 256, Z hi 64 and acc2 in 512 columns
    return kc == 64 ? launch_wide<64>(a, grid, st) : launch_wide<32>(a, grid, st);
  }
  if (zt == 2 && a.mpad > 128) return cudaErrorInvalidValue;   // acc1 twice, Z and acc2 in 512 columns
  if (cg == 2) {
    if (zt == 2) return kc == 64 ? launch_geom<64, 2, 2>(a, grid, st) : launch_geom<32, 2, 2>(a, grid, st);
    return kc == 64 ? launch_geom<64, 1, 2>(a, grid, st) : launch_geom<32, 1, 2>(a, grid, st);
  }
  if (kc == 64)
    return zt == 2 ? launch_geom<64, 2, 1>(a, grid, st)
                   : zt ? launch_geom<64, 1, 1>(a, grid, st) : launch_geom<64, 0, 1>(a, grid, st);
  return zt == 2 ? launch_geom<32, 2, 1>(a, grid, st)
                 : zt ? launch_geom<32, 1, 1>(a, grid, st) : launch_geom<32, 0, 1>(a, grid, st);
}

// device error word shared by all launches (checked by the host after each pass)
int* err_word() {
  static int* p = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    if (cudaMalloc(&p, 16) == cudaSuccess) cudaMemset(p, 0, 16);
    else p = nullptr;
  });
  return p;
}

int sm_count() {
  static int n = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      n = 148;
    }
  });
  return n;
}

int view_kc(const TcView& v) { return (v.kc == 32 || v.kc == 64) ? v.kc : ring_kc(); }
int view_cg(const TcView& v) { return (v.cg == 2 && v.zt != 3) ? 2 : 1; }
int view_zt(const TcView& v) {
  return v.zt == 3 ? 3 : v.zt == 2 ? 2 : (v.zt == 1 || view_cg(v) == 2) ? 1 : 0;
}
// rows of a B box (the CTA's share of a B tile, or a pair of B tiles) and of a chained-operand box
int view_brows(const TcView& v) { return view_zt(v) == 3 ? 256 : 128 / view_cg(v); }
int view_mrows(const TcView& v) { return (int)v.mpad / view_cg(v); }

// grid x extent of a launch over `units` 128-row A tiles: a CTA pair takes two
int64_t tile_grid(const TcView& v, int64_t units) { return view_cg(v) == 2 ? 2 * ceil_div(units, 2) : units; }

cudaError_t common_args(const TcView& v, TcArgs& a) {
  memset(&a, 0, sizeof(a));
  a.nk = (int)(v.dld / view_kc(v));
  a.mpad = (int)v.mpad;
  a.R = v.R;
  a.C = v.C;
  a.nsplit = v.nsplit;
  a.bias = v.bias;
  a.scale = v.scale;
  a.inv_xg = v.inv_xg;
  a.bias_in_mma = v.bias_in_mma;
  a.fslots = v.fslots;
  a.err = err_word();
  if (!a.err) return cudaErrorMemoryAllocation;
  a.timeout_cycles = 4000000000LL;   // about two seconds at the boost clock
  if (v.mpad > 256 || v.C > MAXG) return cudaErrorInvalidValue;   // the host checks these limits first
  return cudaSuccess;
}


}  // namespace

cudaError_t tc_make_map_bf16(CUtensorMap* m, const void* ptr, int64_t cols, int64_t rows, int64_t ld, int box_rows,
                             int kc) {
  return make_map(m, ptr, cols, rows, ld, box_rows, kc);
}

int* tc_error_ptr() { return err_word(); }

cudaError_t tc_wait_probe(long long cycles, cudaStream_t st) {
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.err = err_word();
  if (!a.err) return cudaErrorMemoryAllocation;
  a.timeout_cycles = cycles;
  k_wait_probe<<<1, 32, 0, st>>>(a);
  return cudaGetLastError();
}

int tc_error_word() {
  int h = 0;
  int* p = err_word();
  if (!p) return -1;
  if (cudaMemcpy(&h, p, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  if (h) cudaMemset(p, 0, 4);
  return h;
}

namespace {
cudaError_t write_z(const TcView& v, int64_t r0, int64_t nr, int64_t f0, int64_t nf, float* out, __half* zt_hi,
                    __half* zt_lo, float zt_scale, int64_t ldo) {
  if (nr <= 0 || nf <= 0) return cudaSuccess;
  TcArgs a;
  cudaError_t e = common_args(v, a);
  if (e != cudaSuccess) return e;
  a.mode = MODE_WRITEZ;
  a.a_ok = v.row_ok;
  a.b_ok = v.feat_ok;
  a.wz_r0 = r0; a.wz_nr = nr; a.wz_f0 = f0; a.wz_nf = nf; a.ldo = ldo;
  a.out = out;
  a.zt_hi = zt_hi;
  a.zt_lo = zt_lo;
  a.zt_scale = zt_scale;
  a.out_elems = zt_hi ? (nf - 1) * ldo + nr : (nr - 1) * ldo + nf;
  if ((e = make_map(&a.tA_hi, v.Xhi, v.dld, v.nslots, v.dld, 128, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tA_lo, v.Xlo, v.dld, v.nslots, v.dld, 128, view_kc(v))) != cudaSuccess) return e;
  const int brows = view_brows(v);
  if ((e = make_map(&a.tB_hi, v.Ghi, v.dld, v.fslots, v.dld, brows, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tB_lo, v.Glo, v.dld, v.fslots, v.dld, brows, view_kc(v))) != cudaSuccess) return e;
  a.tM_hi = a.tB_hi;
  a.tM_lo = a.tB_lo;
  return launch(a, dim3((unsigned)tile_grid(v, ceil_div(nr, 128))), v.st, view_kc(v), view_zt(v), view_cg(v));
}
}  // namespace

cudaError_t tc_write_z(const TcView& v, int64_t r0, int64_t nr, int64_t f0, int64_t nf, float* out, int64_t ldo) {
  return write_z(v, r0, nr, f0, nf, out, nullptr, nullptr, 0.f, ldo);
}

cudaError_t tc_write_zt_split(const TcView& v, int64_t r0, int64_t nr, int64_t f0, int64_t nf, float scale,
                              __half* hi, __half* lo, int64_t ldt) {
  return write_z(v, r0, nr, f0, nf, nullptr, hi, lo, scale, ldt);
}

namespace {
// arguments and grid of pass 1 / pass 2 for a view (no launch); `items` receives the pass-2
// work items (row tiles or their pairs times column blocks)
cudaError_t args_pass1(const TcView& v, float* Rpart, TcArgs& a, dim3& grid) {
  cudaError_t e = common_args(v, a);
  if (e != cudaSuccess) return e;
  a.mode = MODE_PASS1;
  a.row_slot = v.d_row_slot; a.row_size = v.d_row_size; a.col_slot = v.d_col_slot; a.col_size = v.d_col_size;
  a.a_ok = v.feat_ok;
  a.b_ok = v.row_ok;
  a.out = Rpart;
  a.out_elems = (int64_t)v.nsplit * v.R * v.fslots * v.mpad;
  a.out_block_stride = v.fslots * v.mpad;
  a.m_amax = v.v_amax;
  a.bmask = v.bmask;
  a.m_shared = v.v_shared;
  const int cg = view_cg(v), brows = view_brows(v), mrows = view_mrows(v);
  if ((e = make_map(&a.tA_hi, v.Ghi, v.dld, v.fslots, v.dld, 128, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tA_lo, v.Glo, v.dld, v.fslots, v.dld, 128, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tB_hi, v.Xhi, v.dld, v.nslots, v.dld, brows, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tB_lo, v.Xlo, v.dld, v.nslots, v.dld, brows, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tM_hi, v.VThi, v.nslots, (int64_t)v.C * v.mpad, v.nslots, mrows, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tM_lo, v.VTlo, v.nslots, (int64_t)v.C * v.mpad, v.nslots, mrows, view_kc(v))) != cudaSuccess) return e;
  // CTA pairs: the feature tiles of every column block in pairs
  int64_t gx = v.fslots / 128;
  if (cg == 2) {
    gx = 0;
    for (int j = 0; j < v.C; ++j) gx += 2 * ceil_div(ceil_div(v.col_size[j], 128), 2);
  }
  grid = dim3((unsigned)gx, (unsigned)v.R, (unsigned)v.nsplit);
  return cudaSuccess;
}

cudaError_t args_pass2(const TcView& v, const __half* Mhi, const __half* Mlo, float* out, const unsigned* m_amax,
                       unsigned* out_amax, TcArgs& a, int64_t& items) {
  cudaError_t e = common_args(v, a);
  if (e != cudaSuccess) return e;
  a.mode = MODE_PASS2;
  a.row_slot = v.d_row_slot; a.row_size = v.d_row_size; a.col_slot = v.d_col_slot; a.col_size = v.d_col_size;
  a.a_ok = v.row_ok;
  a.b_ok = v.feat_ok;
  a.out = out;
  a.out_elems = (int64_t)v.C * v.nslots * v.mpad;
  a.out_block_stride = v.nslots * v.mpad;
  a.m_amax = m_amax;
  a.out_amax = out_amax;
  a.bmask = v.bmask;
  a.nrow_tiles = v.row_tiles > 0 ? std::min<int64_t>(v.row_tiles, v.nslots / 128) : v.nslots / 128;
  const int cg = view_cg(v), brows = view_brows(v), mrows = view_mrows(v);
  if ((e = make_map(&a.tA_hi, v.Xhi, v.dld, v.nslots, v.dld, 128, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tA_lo, v.Xlo, v.dld, v.nslots, v.dld, 128, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tB_hi, v.Ghi, v.dld, v.fslots, v.dld, brows, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tB_lo, v.Glo, v.dld, v.fslots, v.dld, brows, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tM_hi, Mhi, v.fslots, (int64_t)v.R * v.mpad, v.fslots, mrows, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tM_lo, Mlo, v.fslots, (int64_t)v.R * v.mpad, v.fslots, mrows, view_kc(v))) != cudaSuccess) return e;
  // a CTA pair takes items of two row tiles of a block
  int64_t nunits = a.nrow_tiles;
  if (cg == 2) {
    nunits = 0;
    for (int i = 0; i < v.R; ++i) {
      const int64_t end = (i + 1 < v.R) ? v.row_slot[i + 1] : a.nrow_tiles * 128;
      if (end > v.row_slot[i]) nunits += ceil_div((end - v.row_slot[i]) / 128, 2);
    }
  }
  items = nunits * v.C;
  return cudaSuccess;
}
}  // namespace

cudaError_t tc_pass1(const TcView& v, float* Rpart) {
  TcArgs a;
  dim3 grid;
  cudaError_t e = args_pass1(v, Rpart, a, grid);
  if (e != cudaSuccess) return e;
  return launch(a, grid, v.st, view_kc(v), view_zt(v), view_cg(v));
}

cudaError_t tc_pass2(const TcView& v, const __half* Mhi, const __half* Mlo, int64_t m_block_stride,
                     float* out, int per_block, const unsigned* m_amax, unsigned* out_amax) {
  (void)m_block_stride;
  (void)per_block;
  TcArgs a;
  int64_t nitems = 0;
  cudaError_t e = args_pass2(v, Mhi, Mlo, out, m_amax, out_amax, a, nitems);
  if (e != cudaSuccess) return e;
  // persistent: one CTA per SM (the ring fills most of shared memory), enough CTAs that
  // none takes more than MAXG work items
  const int cg = view_cg(v);
  const int maxg = view_zt(v) == 3 ? W_MAXG : MAXG;
  const int64_t grid = std::min<int64_t>(nitems, std::max<int64_t>(sm_count() / cg, ceil_div(nitems, maxg)));
  return launch(a, dim3((unsigned)(grid * cg)), v.st, view_kc(v), view_zt(v), cg);
}

// ------------------------------------------------------------------ several solves, one launch
struct TcMulti {
  MultiArgs m;
  int64_t grid = 0;
  TcArgs* table = nullptr;   // device copy of the solves' arguments
};

void tc_multi_destroy(TcMulti* t) {
  if (!t) return;
  if (t->table) cudaFree(t->table);
  delete t;
}

cudaError_t tc_multi_create(const TcView* views, int n, int which, float* const* outs, const __half* const* Mhi,
                            const __half* const* Mlo, const unsigned* const* m_amax, unsigned* const* out_amax,
                            TcMulti** out) {
  *out = nullptr;
  if (n < 1 || n > MULTI_MAX || (which != 1 && which != 2)) return cudaErrorInvalidValue;
  std::vector<TcArgs> args(n);
  std::vector<int64_t> items(n, 0);
  TcMulti* t = new TcMulti();
  memset(&t->m, 0, sizeof(t->m));
  t->m.ngroups = n;
  cudaError_t e = cudaSuccess;
  for (int g = 0; g < n && e == cudaSuccess; ++g) {
    TcView v = views[g];
    v.kc = 64;   // one kernel instance serves every solve: the default ring, Z in TMEM, one CTA
    v.zt = 1;
    v.cg = 1;
    if (which == 1) {
      dim3 grid;
      e = args_pass1(v, outs[g], args[g], grid);
      t->m.gx[g] = grid.x;
      t->m.gy[g] = (int)grid.y;
      items[g] = (int64_t)grid.x * grid.y * grid.z;
    } else {
      e = args_pass2(v, Mhi[g], Mlo[g], outs[g], m_amax[g], out_amax[g], args[g], items[g]);
    }
  }
  if (e == cudaSuccess && which == 2) {
    // the persistent CTAs of pass 2 shared in proportion to the solves' work items (every
    // item is one 128-row tile against one column block), each solve taking at least one CTA
    // and no CTA more than MAXG items
    int64_t total = 0;
    for (int g = 0; g < n; ++g) total += items[g];
    for (int g = 0; g < n; ++g) {
      const int64_t share = std::max<int64_t>(1, (int64_t)sm_count() * items[g] / std::max<int64_t>(total, 1));
      t->m.gx[g] = std::min<int64_t>(std::max<int64_t>(items[g], 1),
                                     std::max<int64_t>(share, ceil_div(items[g], MAXG)));
      t->m.gy[g] = 1;
    }
  }
  if (e == cudaSuccess) {
    int64_t start = 0;
    for (int g = 0; g < n; ++g) {
      t->m.start[g] = start;
      start += which == 1 ? items[g] : t->m.gx[g];
    }
    t->m.start[n] = start;
    t->grid = start;
    if (start > 0x7fffffffLL) e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) e = cudaMalloc(&t->table, sizeof(TcArgs) * n);
  if (e == cudaSuccess) e = cudaMemcpy(t->table, args.data(), sizeof(TcArgs) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    tc_multi_destroy(t);
    return e;
  }
  t->m.table = t->table;
  *out = t;
  return cudaSuccess;
}

cudaError_t tc_multi_launch(const TcMulti* t, cudaStream_t st) {
  if (!t || t->grid == 0) return cudaSuccess;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_regen_multi<64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_bytes<64, 1, 1>());
  });
  if (attr_err != cudaSuccess) return attr_err;
  k_regen_multi<64, 1><<<(unsigned)t->grid, NTHREADS, smem_bytes<64, 1, 1>(), st>>>(t->m);
  return cudaGetLastError();
}

cudaError_t tc_predict(const TcView& v, const __half* Xh, const __half* Xl, int64_t nrows,
                       const __half* Mhi, const __half* Mlo, const unsigned* m_amax, float* out) {
  if (nrows <= 0) return cudaSuccess;
  if (nrows % 128) return cudaErrorInvalidValue;
  TcArgs a;
  cudaError_t e = common_args(v, a);
  if (e != cudaSuccess) return e;
  a.mode = MODE_PREDICT;
  a.a_rows = nrows;
  a.a_ok = nullptr;
  a.b_ok = v.feat_ok;
  a.out = out;
  a.out_elems = nrows * v.mpad;
  a.m_amax = m_amax;
  const int cg = view_cg(v), brows = view_brows(v), mrows = view_mrows(v);
  if ((e = make_map(&a.tA_hi, Xh, v.dld, nrows, v.dld, 128, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tA_lo, Xl, v.dld, nrows, v.dld, 128, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tB_hi, v.Ghi, v.dld, v.fslots, v.dld, brows, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tB_lo, v.Glo, v.dld, v.fslots, v.dld, brows, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tM_hi, Mhi, v.fslots, v.mpad, v.fslots, mrows, view_kc(v))) != cudaSuccess) return e;
  if ((e = make_map(&a.tM_lo, Mlo, v.fslots, v.mpad, v.fslots, mrows, view_kc(v))) != cudaSuccess) return e;
  return launch(a, dim3((unsigned)tile_grid(v, nrows / 128)), v.st, view_kc(v), view_zt(v), cg);
}

RFF_CHECK_UNIT(tc)

}  // namespace rff
