// dvm_sweep_pair.cuh -- the FP32 row sweep with two velocity groups per warp ("paired groups");
// included by dvm_sweep.cuh, whose helpers it uses.
//
// The same update as sweep_tile (Eq. (iteration), second-order upwind, lagged walls and seams), with
// lane l of a warp holding velocity l of two groups of the same quadrant: every per-velocity value is a
// float2 and every update is a packed FP32x2 FMA (a scalar record field enters both halves as a
// broadcast operand, which costs nothing).  The two groups share the cell records, the waits, the
// staging and the loop control, so those are paid once per 64 velocities.  The ring rows hold the 64
// values interleaved (entry 2l + k is velocity l of the pair's group k), and the per-cell sums are the
// same tensor-core contraction over 64 velocities.  The ring of a warp is twice as wide: each paired
// block lays out its own shared memory (a 256-cell grid, 16 warps at 16 cells per chunk, fits one pair
// per block in 224 of the 227 KB; narrower grids fit several), with one record stage per warp that is
// refilled as soon as the cell loop is done.  FP32 storage, forward sweeps, uniform collision rate;
// rows 0 and 1 of a periodic y axis read their wrapped upstream rows straight from the seam buffers.
#pragma once

namespace dvm {
namespace sweep {

__device__ __forceinline__ float2 bcast(float x) { return make_float2(x, x); }

// B fragment of the interleaved 64 x 6 weight matrix for k-step s and lane ln, as in weight_fragments:
// {hi(k0), hi(k0 + 4), lo(k0), lo(k0 + 4)} of column n = ln / 4, k0 = 8 s + ln % 4.
__device__ __forceinline__ uint4 weight_fragment64(const float *wts, int s, int ln) {
  const int n = ln >> 2, t = ln & 3;
  uint32_t v[4];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float w = n < kSweepWtsRows ? wts[n * kPairRS + 8 * s + t + 4 * e] : 0.f;
    v[e] = tf32_rna(w);
    v[2 + e] = tf32_rna(w - __uint_as_float(v[e]));
  }
  return make_uint4(v[0], v[1], v[2], v[3]);
}

// The chunk's ring tile (16 rows of 64 interleaved velocities) times the weights, as cell_sums_mma; the
// B fragments come from shared memory (bfl: this lane's fragment of k-step 0, k-steps 32 entries apart).
__device__ __forceinline__ void cell_sums_mma64(uint32_t base, const uint4 *bfl, float (&d)[4]) {
  d[0] = d[1] = d[2] = d[3] = 0.f;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    uint32_t a[4], ah[4], al[4];
    ldsm_x4(base + s * 32, a);
    const uint4 b = bfl[s * kLanes];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ah[i] = (a[i] + 0x1000u) & 0xffffe000u;
      al[i] = __float_as_uint(__uint_as_float(a[i]) - __uint_as_float(ah[i]));
    }
    mma_tf32(d, al, b.x, b.y);
    mma_tf32(d, ah, b.z, b.w);
    mma_tf32(d, ah, b.x, b.y);
  }
}

// PER as for sweep_tile: the persistent kernel hands out tiles of active members only (every read of data
// written earlier in the same launch below already goes through L2: cp.async.cg, __ldcg).
template <int CW, bool PER = false>
__device__ __forceinline__ void sweep_tile_pair(const LaunchDesc &L, int map, unsigned char *smem, int Rb) {
  constexpr int RS = kPairRS;
  constexpr int NPC = (int)sizeof(SweepRec<float>) / 16, NPIECE = NPC * CW, PPL = (NPIECE + kLanes - 1) / kLanes;
  const InstanceDesc *__restrict__ D = L.inst + ((map >> 16) & 0x3fff);
  DeviceState *st = D->state;
  if (!PER && *reinterpret_cast<volatile int *>(&st->done)) return;

  const int nx = D->nx, ny = D->ny, ncell = D->ncell;
  const bool px = D->periodic_x != 0, py = D->periodic_y != 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int R = (nx + CW - 1) / CW;  // rows in flight (host ensures ntile R <= the layout's warps)
  const int g0 = map & 0xfff;         // first group of the first pair; pair j is g0 + 2j, g0 + 2j + 1
  const int ntile = max((map >> 12) & 15, 1);
  const int wt = w / R, lw = w - wt * R, wb = wt * R;
  const int ga = g0 + 2 * wt;         // this warp's pair (one quadrant)
  const int quad = min(ga, D->ngroups - 1) / D->groups_per_quadrant;
  const bool xneg = (quad & 1) != 0, yneg = (quad & 2) != 0;

  // this block's own layout (the launch provides the largest any paired block needs)
  const SweepPairSmemLayout SL = sweep_pair_smem_layout(ntile * R, CW, ntile);
  float *ring = reinterpret_cast<float *>(smem + SL.ring);
  SweepRec<float> *stage = reinterpret_cast<SweepRec<float> *>(smem + SL.stage);
  float *invt_all = reinterpret_cast<float *>(smem + SL.inv);
  float *wts_all = reinterpret_cast<float *>(smem + SL.wts);
  uint4 *bfr_all = reinterpret_cast<uint4 *>(smem + SL.bfr);
  int *prog = reinterpret_cast<int *>(smem + SL.prog);

  // zero the layout (ring slots read before being written meet zero coefficients), then the tables
  for (size_t b = threadIdx.x; b < SL.total / 16; b += (size_t)Rb * kLanes)
    reinterpret_cast<float4 *>(smem)[b] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  for (int j = 0; j < ntile; ++j) {
    const float *vA = static_cast<const float *>(D->vel) + (size_t)(g0 + 2 * j) * kNumVelFields * kLanes;
    const float *vB = vA + kNumVelFields * kLanes;
    const float *iA = static_cast<const float *>(D->inv_den) + (size_t)(g0 + 2 * j) * kInvRows * kLanes;
    const float *iB = iA + kInvRows * kLanes;
    for (int i = threadIdx.x; i < kInvRows * 2 * kLanes; i += Rb * kLanes) {
      const int row = i >> 6, e = i & 63;
      invt_all[j * kInvRows * 2 * kLanes + i] = ((e & 1) ? iB : iA)[row * kLanes + (e >> 1)];
    }
    for (int i = threadIdx.x; i < kSweepWtsRows * 2 * kLanes; i += Rb * kLanes) {
      const int m = i >> 6, e = i & 63;
      const int fld = m < 4 ? kW0 + m : (m == 4 ? kWnx : kWny);
      wts_all[(j * kSweepWtsRows + m) * RS + e] = ((e & 1) ? vB : vA)[fld * kLanes + (e >> 1)];
    }
  }
  for (int i = threadIdx.x; i < min(Rb, ntile * R); i += Rb * kLanes) prog[i] = i % R;
  __syncthreads();
  for (int i = threadIdx.x; i < ntile * 8 * kLanes; i += Rb * kLanes) {
    const int j = i / (8 * kLanes), sl = i - j * 8 * kLanes;
    bfr_all[i] = weight_fragment64(wts_all + j * kSweepWtsRows * kPairRS, sl >> 5, sl & 31);
  }
  __syncthreads();
  if (wt >= ntile) return;

  const float *vA = static_cast<const float *>(D->vel) + (size_t)ga * kNumVelFields * kLanes;
  const float *vB = vA + kNumVelFields * kLanes;
  auto pairv = [&](int fld) { return make_float2(vA[fld * kLanes + lane], vB[fld * kLanes + lane]); };
  const float2 v1 = pairv(kV1), v2 = pairv(kV2), em1 = pairv(kE2m1), cx = pairv(kCx), cy = pairv(kCy);
  const float *invt_lane2 = invt_all + wt * kInvRows * 2 * kLanes + 2 * lane;
  const float sshift = __ldcg(&st->s);
  const SweepRec<float> *__restrict__ rec = static_cast<const SweepRec<float> *>(D->rec) + (size_t)quad * ncell;
  // the pair's second group sits one group further in each per-group array (offsets, not pointers:
  // registers are scarce)
  float *seamxA = static_cast<float *>(D->seam_x) + (size_t)ga * ny * 2 * kLanes;
  float *seamyA = static_cast<float *>(D->seam_y) + (size_t)ga * nx * 2 * kLanes;
  float *houtA = D->h ? static_cast<float *>(D->h) + (size_t)ga * ncell * kLanes : nullptr;
  const int sxo = ny * 2 * kLanes, syo = nx * 2 * kLanes;
  double *acc = D->acc;
  double *facc = D->facc + (size_t)((__ldcg(&st->iter) + 1) & 1) * ncell * 4;
  const int sidex = xneg ? kW : kE, sidey = yneg ? kS : kN;
  const int wprev = wb + (lw + R - 1) % R, wnext2 = wb + (lw + 2) % R;
  // per-cell sums: ldmatrix row and destinations of the lane's two result columns
  const uint4 *bfl = bfr_all + wt * 8 * kLanes + lane;
  const int t4 = lane & 3, g4 = lane >> 2;
  const uint32_t ldsm_off = (uint32_t)((min((lane & 7) + 8 * ((lane >> 3) & 1), CW - 1) * RS + 4 * (lane >> 4)) * 4);
  double *const red_base = t4 == 2 ? facc : acc;
  double *const red_p0 = red_base + (t4 == 2 ? sidex : 2 * t4);
  double *const red_p1 = red_base + (t4 == 2 ? sidey : 2 * t4 + 1);
  uint32_t red_am0 = kSolid, red_cv0 = 0u, red_am1 = kSolid, red_cv1 = 0u;
  if (t4 == 2) {
    red_am0 = red_cv0 = kIncX;
    red_am1 = red_cv1 = kIncY;
  } else if (t4 == 3) {
    red_am0 = red_am1 = 0u;
    red_cv0 = red_cv1 = 1u;
  }
  // record staging of a full chunk (as in sweep_tile)
  int st_dst[PPL];
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int pc = lane + k * kLanes, r = pc / NPC, l = xneg ? CW - 1 - r : r;
    st_dst[k] = l * (int)sizeof(SweepRec<float>) + 16 * (pc - r * NPC);
  }
  float2 pf_hp1 = bcast(0.f), pf_hp2 = bcast(0.f);
  // records of chunk (q, c) into the warp's stage (one buffer: the next chunk is staged as soon as the
  // cell loop of the current one is done, overlapping the copy with its sums and the next wait)
  auto issue = [&](int q, int c) {
    const int j = yneg ? ny - 1 - q : q;
    SweepRec<float> *sdst = stage + (size_t)w * CW;
    const int p0 = c * CW;
    const int cnt = min(CW, nx - p0);
    const char *src = reinterpret_cast<const char *>(rec + j * nx + (xneg ? nx - p0 - cnt : p0));
    if (cnt == CW) {
#pragma unroll
      for (int k = 0; k < PPL; ++k)
        if (NPIECE % kLanes == 0 || lane + k * kLanes < NPIECE)
          cp_async16(reinterpret_cast<char *>(sdst) + st_dst[k], src + 16 * (lane + k * kLanes));
    } else {
      for (int pc = lane; pc < NPC * cnt; pc += kLanes) {
        const int r = pc / NPC, l = xneg ? cnt - 1 - r : r;
        cp_async16(reinterpret_cast<char *>(sdst + l) + 16 * (pc - r * NPC), src + 16 * pc);
      }
      if (lane >= cnt && lane < CW) {
        float4 *dst = reinterpret_cast<float4 *>(sdst + lane);
#pragma unroll
        for (int b = 0; b < NPC; ++b) dst[b] = make_float4(0.f, 0.f, 0.f, 0.f);
        sdst[lane].code = kSolid | (9u << kInvShift);
      }
    }
    if (c == 0 && px) {
      // x-seam values of the new row: columns nx-1 (slot 1) and nx-2 (slot 0) of the last sweep
      const float *sx = seamxA + j * 2 * kLanes + lane;
      pf_hp1 = make_float2(__ldcg(sx + kLanes), __ldcg(sx + sxo + kLanes));
      pf_hp2 = make_float2(__ldcg(sx), __ldcg(sx + sxo));
    }
    cp_async_commit();
  };

  // one chunk: MODE 0 upstream rows from the ring; MODE 1 (row 0 of a periodic y axis) both wrapped rows
  // from the seam buffers; MODE 2 (row 1) row q-1 from the ring, row q-2 from the seam buffers
  float2 hp1 = bcast(0.f), hp2 = bcast(0.f), row_hp1 = bcast(0.f), row_hp2 = bcast(0.f);
  auto run_chunk = [&](auto mode_tag, int q, int c, int t, const SweepRec<float> *rs, float *myr, const float *pr1,
                       const float *pr2, int nq, int nc) {
    constexpr int MODE = decltype(mode_tag)::value;
    const int j = yneg ? ny - 1 - q : q;
    if (c == 0) {
      hp1 = px ? make_float2(row_hp1.x - sshift, row_hp1.y - sshift) : bcast(0.f);
      hp2 = px ? make_float2(row_hp2.x - sshift, row_hp2.y - sshift) : bcast(0.f);
    }
    const int p0 = c * CW;
    const int cnt = min(CW, nx - p0);
    constexpr int SUB = CW < 4 ? CW : 4;
#pragma unroll
    for (int l0 = 0; l0 < CW; l0 += SUB) {
      float2 base[SUB], invv[SUB];
      float cax1[SUB], cax2[SUB], cxw[SUB];
#pragma unroll
      for (int u = 0; u < SUB; ++u) {
        const int l = l0 + u;
        const SweepRec<float> r = rs[l];
        float2 hq1, hq2;
        if (MODE == 0) {
          hq1 = *reinterpret_cast<const float2 *>(pr1 + l * RS + 2 * lane);
          hq2 = *reinterpret_cast<const float2 *>(pr2 + l * RS + 2 * lane);
        } else {
          const int i = xneg ? nx - 1 - (p0 + l) : p0 + l;
          const size_t o = (size_t)max(0, min(i, nx - 1)) * 2 * kLanes + lane;
          const bool in = l < cnt;
          const float *sy = seamyA + o;
          if (MODE == 1)
            hq1 = in ? make_float2(__ldcg(sy + kLanes) - sshift, __ldcg(sy + syo + kLanes) - sshift) : bcast(0.f);
          else
            hq1 = *reinterpret_cast<const float2 *>(pr1 + l * RS + 2 * lane);
          const float *s2 = MODE == 1 ? sy : sy + kLanes;
          hq2 = in ? make_float2(__ldcg(s2) - sshift, __ldcg(s2 + syo) - sshift) : bcast(0.f);
        }
        const float2 Rk = __ffma2_rn(bcast(r.D), em1, __ffma2_rn(bcast(r.C), v2, __ffma2_rn(bcast(r.B), v1, bcast(r.A))));
        const float2 by = __ffma2_rn(bcast(r.ay1), hq1, __ffma2_rn(bcast(r.ay2), hq2, bcast(r.yw)));
        base[u] = __ffma2_rn(cy, by, Rk);
        // 1/denominator row (code >> kInvShift) & 15 of the pair's table: 256-byte rows
        invv[u] = *reinterpret_cast<const float2 *>(reinterpret_cast<const char *>(invt_lane2) +
                                                    ((r.code & (15u << kInvShift)) << 1));
        cax1[u] = r.ax1;
        cax2[u] = r.ax2;
        cxw[u] = r.xw;
      }
#pragma unroll
      for (int u = 0; u < SUB; ++u) {
        const float2 bx = __ffma2_rn(bcast(cax1[u]), hp1, __ffma2_rn(bcast(cax2[u]), hp2, bcast(cxw[u])));
        const float2 h = __fmul2_rn(__ffma2_rn(cx, bx, base[u]), invv[u]);
        hp2 = hp1;
        hp1 = h;
        *reinterpret_cast<float2 *>(myr + (l0 + u) * RS + 2 * lane) = h;
      }
    }
    __syncwarp();
    if (lane == 0) st_release(&prog[w], t + 1);
    // the codes the sums need, then the stage is free for the next chunk
    const uint32_t code0 = g4 < cnt ? rs[g4].code : kSolid;
    const uint32_t code1 = (CW > 8 && g4 + 8 < cnt) ? rs[g4 + 8].code : kSolid;
    __syncwarp();
    if (nq < ny) issue(nq, nc);
    else cp_async_commit();
    if (houtA) {
      for (int l = 0; l < cnt; ++l) {
        const int i = xneg ? nx - 1 - (p0 + l) : p0 + l;
        const float2 h = *reinterpret_cast<const float2 *>(myr + l * RS + 2 * lane);
        houtA[(size_t)(j * nx + i) * kLanes + lane] = h.x;
        houtA[(size_t)ncell * kLanes + (size_t)(j * nx + i) * kLanes + lane] = h.y;
      }
    }
    if (px && p0 + cnt > nx - 2) {
      for (int p = max(p0, nx - 2); p < p0 + cnt; ++p) {
        const float2 h = *reinterpret_cast<const float2 *>(myr + (p - p0) * RS + 2 * lane);
        seamxA[(j * 2 + (p - (nx - 2))) * kLanes + lane] = h.x;
        seamxA[sxo + (j * 2 + (p - (nx - 2))) * kLanes + lane] = h.y;
      }
    }
    if (py && q >= ny - 2) {
      for (int l = 0; l < cnt; ++l) {
        const int i = xneg ? nx - 1 - (p0 + l) : p0 + l;
        const float2 h = *reinterpret_cast<const float2 *>(myr + l * RS + 2 * lane);
        seamyA[(i * 2 + (q - (ny - 2))) * kLanes + lane] = h.x;
        seamyA[syo + (i * 2 + (q - (ny - 2))) * kLanes + lane] = h.y;
      }
    }
    {
      float d[4];
      cell_sums_mma64(smem_u32(myr) + ldsm_off, bfl, d);
      const int e0 = (j * nx + (xneg ? nx - 1 - p0 - g4 : p0 + g4)) * 4;
      const int de = xneg ? -32 : 32;
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        if ((hf == 0 || CW > 8) && g4 + 8 * hf < cnt) {
          const uint32_t code = hf ? code1 : code0;
          const int e = e0 + hf * de;
          if ((code & red_am0) == red_cv0) red_add(red_p0 + e, static_cast<double>(d[2 * hf]));
          if ((code & red_am1) == red_cv1) red_add(red_p1 + e, static_cast<double>(d[2 * hf + 1]));
        }
      }
    }
  };

  auto give_up = [&]() {
    cp_async_wait<0>();
    atomicExch(&st->err_flag, 1);
  };

  int s0 = lw % 3;  // ring slot of the current step t: the warp's steps are lw, lw + 1, ...
  float *ring_w = ring + (size_t)w * 3 * CW * RS;
  const float *ring_p1 = ring + (size_t)wprev * 3 * CW * RS;
  const float *ring_p2 = ring + (size_t)(wb + (lw + 2 * R - 2) % R) * 3 * CW * RS;
  issue(lw, 0);
  for (int q = lw; q < ny; q += R) {
    for (int c = 0; c < R; ++c) {
      const int t = q + c;
      if (c == 0) {
        row_hp1 = pf_hp1;
        row_hp2 = pf_hp2;
      }
      const int nq = (c + 1 < R) ? q : q + R, nc = (c + 1 < R) ? c + 1 : 0;
      cp_async_wait<0>();
      __syncwarp();
      // row q-1 finished this chunk, and row q+2 has read the ring slot written three steps ago
      if (R > 1 && !wait_at_least(&prog[wprev], t)) return give_up();
      if (R > 2 && !wait_at_least(&prog[wnext2], t)) return give_up();
      const SweepRec<float> *rs = stage + (size_t)w * CW;
      const int s1 = s0 == 0 ? 2 : s0 - 1, s2 = s0 == 2 ? 0 : s0 + 1;
      float *myr = ring_w + s0 * (CW * RS);
      const float *pr1 = ring_p1 + s1 * (CW * RS);
      const float *pr2 = ring_p2 + s2 * (CW * RS);
      s0 = s2;
      if (py && q < 2) {
        if (q == 0) run_chunk(std::integral_constant<int, 1>(), q, c, t, rs, myr, pr1, pr2, nq, nc);
        else run_chunk(std::integral_constant<int, 2>(), q, c, t, rs, myr, pr1, pr2, nq, nc);
      } else {
        run_chunk(std::integral_constant<int, 0>(), q, c, t, rs, myr, pr1, pr2, nq, nc);
      }
      __syncwarp();
    }
  }
  if (lane == 0) st_release(&prog[w], INT_MAX / 2);  // no more rows: never wait on this warp again
}

}  // namespace sweep
}  // namespace dvm
