// Block-RHS local solves on the 5th-generation tensor cores: Y_i = C_i X_i
// for every subdomain, C_i = (I - xi_i) A_i^-1 the part of the split local
// inverse (Sec. 2, eq. "inverseBw") stored in bfloat16, X_i the restricted
// residuals of up to 16 right-hand sides, float32 accumulation.
//
// Storage: C_i as the lower triangle of 128x128 super-tiles (diagonal
// super-tiles in full), each super-tile in the canonical 128-byte-swizzled
// K-major shared-memory layout of tcgen05 operands (two 16 KB halves of 64
// columns; row r at r * 128 B, 16-byte chunk j stored at chunk j ^ (r % 8)).
// A plain bulk copy therefore lands a ready operand in shared memory, and the
// same bytes read through an MN-major descriptor are the transposed tile.
//
// One CTA owns whole subdomains (longest-processing-time order).  Per
// subdomain all 128-row blocks of Y accumulate in TMEM (16 float32 columns
// per block, at most 16 blocks = 256 columns), so the symmetric product
// needs no partial sums in memory:
//   super-tile S = C(I, J), J <= I:  Y_I += S X_J  and, for J < I,
//   Y_J += S^T X_I  (M = 128, N = 16, K = 128 as eight K = 16 instructions).
// Warp 4 streams super-tiles through 4 stages with cp.async.bulk on
// mbarriers; thread 0 issues the MMAs and commits each stage back to the
// producer; warps 0-3 stage X in bfloat16 and read Y out of TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <queue>

#include "setup.hpp"

namespace geneo {

namespace {

constexpr int kSt = 128;                          // super-tile edge
constexpr int kStBytes = kSt * kSt * 2;           // 32 KB of bfloat16
constexpr int kTcStages = 4;
constexpr int kTcN = 16;                          // MMA N: right-hand sides, zero padded
constexpr int kXBlockBytes = kSt * kTcN * 2;      // X block: 128 K x 16 N bfloat16 = 4 KB
constexpr int kTmemCols = kTcMaxBlocks * kTcN;    // 256
constexpr int kTcThreads = 160;                   // warps 0-3: X / MMA / epilogue, warp 4: copies
constexpr int kSmemStages = kTcStages * kStBytes;
constexpr int kSmemX = kTcMaxBlocks * kXBlockBytes;
constexpr int kSmemGuard = 8192;  // reads of a misdescribed operand stay inside the allocation
constexpr int kSmemBars = 256;
constexpr size_t kTcSmem = 1024 + kSmemStages + kSmemX + kSmemGuard + kSmemBars;

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tc_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool tc_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 "
      "%0, 1, 0, p;\n}" : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
// bounded: about two seconds of polling
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!tc_try_wait(bar, parity))
    if (clock64() - t0 > 4000000000LL) return false;
  return true;
}

// shared-memory matrix descriptor (tcgen05): start, leading and stride byte
// offsets in 16-byte units, descriptor version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor, kind::f16: D float32, A and B bfloat16, N = 16,
// M = 128; a_mn selects an MN-major (transposed) A operand
__host__ __device__ constexpr uint32_t idesc(bool a_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((uint32_t)(kTcN >> 3) << 17) |
         ((uint32_t)(kSt >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(id), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

// Y_i = C_i X_i for the subdomains listed for this CTA
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_symm(const uint16_t *__restrict__ st, const int64_t *__restrict__ st_off,
              const int32_t *__restrict__ nblk, const int64_t *__restrict__ voff,
              const int32_t *__restrict__ rows, const int32_t *__restrict__ sub_list,
              const int32_t *__restrict__ cta_off, const double *__restrict__ x,
              double *__restrict__ y, int64_t vlen, int k, int *err) {
  extern __shared__ unsigned char smraw[];
  const uint32_t raw = su32(smraw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment
  unsigned char *sm = smraw + (base - raw);
  const uint32_t s_stage = base, s_x = base + kSmemStages;
  const uint32_t s_bar = s_x + kSmemX + kSmemGuard;
  // barriers: full[4], empty[4], done; then the TMEM address and the abort flag
  const uint32_t b_full = s_bar, b_empty = s_bar + 8 * kTcStages, b_done = s_bar + 16 * kTcStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kSmemStages + kSmemX + kSmemGuard +
                                                     16 * kTcStages + 8);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  unsigned char *xs = sm + kSmemStages;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s0 = cta_off[blockIdx.x], s1 = cta_off[blockIdx.x + 1];
  if (tid == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      tc_mbar_init(b_full + 8 * i, 1);
      tc_mbar_init(b_empty + 8 * i, 1);
    }
    tc_mbar_init(b_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    // ---- producer: every super-tile of every subdomain of this CTA, in order
    if (lane == 0) {
      long long g = 0;
      bool ok = true;
      for (int q = s0; q < s1 && ok; ++q) {
        const int m = sub_list[q];
        const int64_t nt = (int64_t)nblk[m] * (nblk[m] + 1) / 2;
        const uint16_t *src = st + st_off[m] * (kStBytes / 2);
        for (int64_t t = 0; t < nt; ++t, ++g) {
          const int sidx = (int)(g % kTcStages);
          if (g >= kTcStages) {
            if (*abort_flag || !tc_wait(b_empty + 8 * sidx, (uint32_t)(((g / kTcStages) - 1) & 1))) {
              *abort_flag = 1;
              atomicCAS(err, kDevOk, kDevTimeout);
              ok = false;
              break;
            }
          }
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                           b_full + 8 * sidx),
                       "r"(kStBytes)
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
              "[%3];" ::"r"(s_stage + sidx * kStBytes),
              "l"(src + t * (kStBytes / 2)), "r"(kStBytes), "r"(b_full + 8 * sidx)
              : "memory");
        }
      }
      // copies issued but never consumed (abort) complete before the CTA ends
      if (!ok) {
        const long long lo = g > kTcStages ? g - kTcStages : 0;
        for (long long h = lo; h < g; ++h)
          tc_wait(b_full + 8 * (int)(h % kTcStages), (uint32_t)((h / kTcStages) & 1));
      }
    }
  } else {
    // ---- warps 0-3
    long long g = 0;  // super-tile counter, as the producer's
    for (int q = s0; q < s1; ++q) {
      const int m = sub_list[q], nb = nblk[m], nrow = rows[m];
      const int64_t vb = voff[m];
      // X in bfloat16, B operand layout: block I at I * 4 KB, K half h at
      // h * 2 KB, row n (right-hand side) at n * 128 B, chunk swizzle n % 8
      for (int e = tid; e < nb * kTcN * kSt; e += 128) {
        const int r = e % kSt, n = (e / kSt) % kTcN, I = e / (kSt * kTcN);
        const int row = I * kSt + r;
        const double v = (n < k && row < nrow) ? x[(int64_t)n * vlen + vb + row] : 0.0;
        const int kk = r & 63;
        const uint32_t off = I * kXBlockBytes + (r >> 6) * 2048 + n * 128 +
                             ((((kk >> 3) ^ (n & 7)) << 4) | ((kk & 7) << 1));
        *reinterpret_cast<__nv_bfloat16 *>(xs + off) = __double2bfloat16(v);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int I = 0; I < nb && !*abort_flag; ++I) {
          for (int J = 0; J <= I; ++J, ++g) {
            const int sidx = (int)(g % kTcStages);
            if (!tc_wait(b_full + 8 * sidx, (uint32_t)((g / kTcStages) & 1))) {
              *abort_flag = 1;
              atomicCAS(err, kDevOk, kDevTimeout);
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = s_stage + sidx * kStBytes;
            // Y_I += S X_J: A K-major (K halves at +16 KB), B = X_J
            for (int s = 0; s < kSt / 16; ++s) {
              const uint32_t ka = a0 + (s >> 2) * 16384 + (s & 3) * 32;
              const uint32_t kb = s_x + J * kXBlockBytes + (s >> 2) * 2048 + (s & 3) * 32;
              mma_bf16(tmem + I * kTcN, sdesc(ka, 16384, 1024), sdesc(kb, 2048, 1024),
                       idesc(false), (J > 0 || s > 0) ? 1u : 0u);
            }
            if (J < I) {
              // Y_J += S^T X_I: the same bytes as an MN-major A (M halves at
              // +16 KB, K groups of 8 rows at +1 KB)
              for (int s = 0; s < kSt / 16; ++s) {
                const uint32_t ka = a0 + s * 2048;
                const uint32_t kb = s_x + I * kXBlockBytes + (s >> 2) * 2048 + (s & 3) * 32;
                mma_bf16(tmem + J * kTcN, sdesc(ka, 16384, 1024), sdesc(kb, 2048, 1024),
                         idesc(true), 1u);
              }
            }
            mma_commit(b_empty + 8 * sidx);
          }
        }
        // completes once every MMA issued so far has finished
        mma_commit(b_done);
      }
      __syncwarp();
      const uint32_t dpar = (uint32_t)((q - s0) & 1);
      if (!tc_wait(b_done, dpar)) {
        *abort_flag = 1;
        atomicCAS(err, kDevOk, kDevTimeout);
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      __syncwarp();
      // warp-uniform decision before the warp-collective TMEM loads
      if (!__any_sync(0xffffffffu, *abort_flag != 0)) {
        // epilogue: warp w holds TMEM lanes (rows) 32w .. 32w + 31
        const int r = warp * 32 + lane;
        for (int I = 0; I < nb; ++I) {
          uint32_t v[16];
          const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + I * kTcN;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
              "%10, %11, %12, %13, %14, %15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(ta)
              : "memory");
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          const int row = I * kSt + r;
          if (row < nrow)
            for (int n = 0; n < k; ++n)
              y[(int64_t)n * vlen + vb + row] = (double)__uint_as_float(v[n]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// bfloat16 super-tiles from the float32 64-tile storage of C_i (rows and
// columns past the padded dimension are zero); one CTA per super-tile
__global__ void k_pack_bf16(const float *__restrict__ src, const int64_t *__restrict__ toff,
                            const int32_t *__restrict__ nt64, const int32_t *__restrict__ st_sub,
                            const int32_t *__restrict__ st_I, const int32_t *__restrict__ st_J,
                            uint16_t *__restrict__ dst) {
  const int64_t q = blockIdx.x;
  const int m = st_sub[q], I = st_I[q], J = st_J[q];
  const int64_t dim = (int64_t)nt64[m] * kTile;
  unsigned char *d = reinterpret_cast<unsigned char *>(dst + q * (kStBytes / 2));
  for (int e = threadIdx.x; e < kSt * kSt; e += blockDim.x) {
    const int r = e / kSt, cc = e % kSt;
    const int64_t R = (int64_t)I * kSt + r, Cc = (int64_t)J * kSt + cc;
    float v = 0.f;
    if (R < dim && Cc < dim) {
      const int64_t a = R >= Cc ? R : Cc, b = R >= Cc ? Cc : R;
      const int64_t ti = a / kTile, tj = b / kTile;
      const float t = src[(toff[m] + ti * (ti + 1) / 2 + tj) * kTileElems +
                          (a % kTile) * kTile + (b % kTile)];
      // the float32 storage keeps the identity on its padding rows; the
      // padded part of C_i is zero here
      v = t;
    }
    const int h = cc >> 6, kk = cc & 63;
    const uint32_t off = h * 16384 + r * 128 + ((((kk >> 3) ^ (r & 7)) << 4) | ((kk & 7) << 1));
    *reinterpret_cast<__nv_bfloat16 *>(d + off) = __float2bfloat16_rn(v);
  }
}

}  // namespace

struct TcFactors {
  int nsub = 0, nctas = 0;
  int64_t nst = 0;
  DevBuf<uint16_t> st;
  DevBuf<int64_t> st_off, voff;
  DevBuf<int32_t> nblk, rows, sub_list, cta_off;
  int64_t bytes() const { return st.bytes(); }
};

void TcDeleter::operator()(TcFactors *t) const { delete t; }

bool tc_supported(const geneo_ctx *c) {
  for (int i = 0; i < c->dec.nsub; ++i)
    if ((c->loc.nt[i] * (int64_t)kTile + kSt - 1) / kSt > kTcMaxBlocks) return false;
  return true;
}

void build_bf16_factors(geneo_ctx *c) {
  cudaStream_t s = c->stream;
  if (!c->loc_f32.p) throw Error(GENEO_ERR_STATE, "internal: bfloat16 factors need the split");
  if (!tc_supported(c))
    throw Error(GENEO_ERR_INVALID_ARG,
                "bfloat16 tensor-core local solves need every subdomain to have at most 2048 "
                "local unknowns");
  auto T = new TcFactors();
  c->tc.reset(T);
  const int nsub = c->dec.nsub;
  T->nsub = nsub;
  std::vector<int32_t> nb(nsub), rows(nsub), sI, sJ, ssub;
  std::vector<int64_t> off(nsub + 1, 0), voff(nsub);
  for (int m = 0; m < nsub; ++m) {
    rows[m] = c->loc.nt[m] * kTile;  // padded local vector length
    nb[m] = (rows[m] + kSt - 1) / kSt;
    voff[m] = c->loc.voff[m];
    off[m + 1] = off[m] + (int64_t)nb[m] * (nb[m] + 1) / 2;
    for (int I = 0; I < nb[m]; ++I)
      for (int J = 0; J <= I; ++J) {
        ssub.push_back(m);
        sI.push_back(I);
        sJ.push_back(J);
      }
  }
  T->nst = off[nsub];
  T->st.alloc(T->nst * (kStBytes / 2));
  {
    DevBuf<int32_t> d_sub, d_I, d_J;
    d_sub.upload(ssub, s);
    d_I.upload(sI, s);
    d_J.upload(sJ, s);
    if (T->nst)
      k_pack_bf16<<<(unsigned)T->nst, 256, 0, s>>>(c->loc_f32.p, c->loc.d_toff.p, c->loc.d_nt.p,
                                                   d_sub.p, d_I.p, d_J.p, T->st.p);
    GENEO_CHECK_LAUNCH();
    GENEO_CUDA(cudaStreamSynchronize(s));
  }
  // longest-processing-time assignment of subdomains to persistent CTAs
  int dev = 0, sms = 0;
  GENEO_CUDA(cudaGetDevice(&dev));
  GENEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int nctas = std::max(1, std::min(sms, nsub));
  std::vector<int> order(nsub);
  for (int m = 0; m < nsub; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
  using Load = std::pair<int64_t, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
  for (int q = 0; q < nctas; ++q) pq.push({0, q});
  std::vector<std::vector<int32_t>> per(nctas);
  for (int m : order) {
    Load l = pq.top();
    pq.pop();
    per[l.second].push_back(m);
    pq.push({l.first + (off[m + 1] - off[m]), l.second});
  }
  std::vector<int32_t> list, coff(1, 0);
  for (auto &v : per) {
    list.insert(list.end(), v.begin(), v.end());
    coff.push_back((int32_t)list.size());
  }
  T->nctas = nctas;
  T->st_off.upload(std::vector<int64_t>(off.begin(), off.end() - 1), s);
  T->voff.upload(voff, s);
  T->nblk.upload(nb, s);
  T->rows.upload(rows, s);
  T->sub_list.upload(list, s);
  T->cta_off.upload(coff, s);
  GENEO_CUDA(cudaFuncSetAttribute(k_tc_symm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kTcSmem));
  GENEO_CUDA(cudaStreamSynchronize(s));
}

int64_t tc_factor_bytes(const geneo_ctx *c) { return c->tc ? c->tc->bytes() : 0; }

void tc_symm(geneo_ctx *c, const double *xl, double *yl, int k, cudaStream_t s, cudaEvent_t e0,
             cudaEvent_t e1) {
  TcFactors &T = *c->tc;
  if (k < 1 || k > kTcN) throw Error(GENEO_ERR_INVALID_ARG, "1..16 right-hand sides");
  if (e0) record_event(e0, s);
  k_tc_symm<<<T.nctas, kTcThreads, kTcSmem, s>>>(T.st.p, T.st_off.p, T.nblk.p, T.voff.p, T.rows.p,
                                                 T.sub_list.p, T.cta_off.p, xl, yl, c->loc.vlen, k,
                                                 c->d_err.p);
  if (e1) record_event(e1, s);
  GENEO_CHECK_LAUNCH();
}

}  // namespace geneo
