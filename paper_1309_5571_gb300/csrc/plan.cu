// Plan creation: operation records of Sec. 7 and the FP64 GEMM work lists.
//
// Sec. 7 observes that the operator blocks A and B are fixed during the Davidson
// iterations, so everything that depends only on them is prepared once: the list of
// operation records (one per transition pair of Eq. 11, each with its input segment,
// output segment, blocks and FLOP workload -- Algorithm 5, line 1), the choice of the
// cheaper multiplication order per record, the device copies of the blocks and the
// diagonal of H_SB used by the Davidson correction.  The paper's CPU/GPU partitioning
// and stream scheduling (Algorithms 5-7) have no counterpart: all records run on the
// GPU in two launches (stage 1: intermediates, stage 2: output GEMMs whose K dimension
// concatenates every record that writes the same output segment).
#include <algorithm>
#include <cstring>
#include <map>

#include "internal.h"

using namespace dmrg;

namespace {

// Operators of one side (left or right), validated against that side's sector dimensions
// and laid out in the host arena (row-major, ld = cols, 256-byte aligned blocks); the data
// is copied by copy_ops once the arena exists.
dmrg_status layout_ops(int nops, const dmrg_operator* ops, const std::vector<int64_t>& dim,
                       std::vector<std::vector<HostBlock>>& dst, size_t* total) {
  const int nsec = (int)dim.size();
  dst.assign(nops, {});
  for (int o = 0; o < nops; ++o) {
    if (ops[o].nblocks < 0 || (ops[o].nblocks && !ops[o].blocks)) {
      set_error("operator %d has a bad block list", o);
      return DMRG_ERR_INVALID_ARG;
    }
    std::map<std::pair<int, int>, int> keys;
    for (int b = 0; b < ops[o].nblocks; ++b) {
      const dmrg_block& blk = ops[o].blocks[b];
      if (blk.idx_in < 0 || blk.idx_in >= nsec || blk.idx_out < 0 || blk.idx_out >= nsec) {
        set_error("operator %d block %d: sector index out of range", o, b);
        return DMRG_ERR_INVALID_ARG;
      }
      if (blk.rows != dim[blk.idx_out] || blk.cols != dim[blk.idx_in] || blk.ld < blk.cols ||
          (blk.rows * blk.cols > 0 && !blk.data)) {
        set_error("operator %d block %d (%d->%d): shape %lldx%lld (ld %lld) does not match "
                  "sectors %lldx%lld",
                  o, b, blk.idx_in, blk.idx_out, (long long)blk.rows, (long long)blk.cols,
                  (long long)blk.ld, (long long)dim[blk.idx_out], (long long)dim[blk.idx_in]);
        return DMRG_ERR_SHAPE;
      }
      if (!keys.emplace(std::make_pair(blk.idx_in, blk.idx_out), b).second) {
        set_error("operator %d has two blocks %d->%d", o, blk.idx_in, blk.idx_out);
        return DMRG_ERR_SHAPE;
      }
      HostBlock hb{blk.idx_in, blk.idx_out, blk.rows, blk.cols, (int64_t)*total};
      dst[o].push_back(hb);
      *total += (size_t)round_up(blk.rows * blk.cols, 32);  // 256-byte aligned blocks
    }
  }
  return DMRG_OK;
}

dmrg_status copy_ops(int nops, const dmrg_operator* ops, const std::vector<std::vector<HostBlock>>& lay,
                     int location, dmrg_plan* p) {
  for (int o = 0; o < nops; ++o) {
    for (int b = 0; b < ops[o].nblocks; ++b) {
      const dmrg_block& blk = ops[o].blocks[b];
      double* out = p->arena_host.data() + lay[o][b].arena_off;
      if (blk.rows * blk.cols == 0) continue;
      if (location == DMRG_HOST_DATA) {
        for (int64_t r = 0; r < blk.rows; ++r)
          std::memcpy(out + r * blk.cols, blk.data + r * blk.ld, sizeof(double) * blk.cols);
      } else {
        DMRG_CUDA_TRY(cudaMemcpy2D(out, sizeof(double) * blk.cols, blk.data,
                                   sizeof(double) * blk.ld, sizeof(double) * blk.cols,
                                   blk.rows, cudaMemcpyDeviceToHost));
      }
    }
  }
  return DMRG_OK;
}

// pair list (i, k) into sectors of p->dimL x p->dimR; segment offsets and n
dmrg_status set_pairs(dmrg_plan* p, int npairs, const int32_t* pi, const int32_t* pk) {
  const int nL = (int)p->dimL.size(), nR = (int)p->dimR.size();
  p->pair_i.assign(pi, pi + npairs);
  p->pair_k.assign(pk, pk + npairs);
  p->pair_off.assign(npairs + 1, 0);
  std::map<std::pair<int, int>, int> seen;
  for (int q = 0; q < npairs; ++q) {
    int i = p->pair_i[q], k = p->pair_k[q];
    if (i < 0 || i >= nL || k < 0 || k >= nR) {
      set_error("pair %d = (%d,%d) out of range", q, i, k);
      return DMRG_ERR_INVALID_ARG;
    }
    if (!seen.emplace(std::make_pair(i, k), q).second) {
      set_error("pair (%d,%d) listed twice", i, k);
      return DMRG_ERR_SHAPE;
    }
    p->pair_off[q + 1] = p->pair_off[q] + p->dimL[i] * p->dimR[k];
  }
  p->n = p->pair_off[npairs];
  return DMRG_OK;
}

dmrg_status validate_and_copy(const dmrg_superblock_desc* d, dmrg_plan* p) {
  if (!d) {
    set_error("desc is NULL");
    return DMRG_ERR_INVALID_ARG;
  }
  if (d->nL <= 0 || d->nR <= 0 || d->npairs < 0 || d->nterms < 0 || d->nopsL < 0 ||
      d->nopsR < 0) {
    set_error("negative or zero sector/pair/term counts");
    return DMRG_ERR_INVALID_ARG;
  }
  if (!d->dimL || !d->dimR || (d->npairs && (!d->pair_i || !d->pair_k)) ||
      (d->nterms && !d->terms) || (d->nopsL && !d->opsL) || (d->nopsR && !d->opsR)) {
    set_error("NULL array in desc");
    return DMRG_ERR_INVALID_ARG;
  }
  if (d->data_location != DMRG_HOST_DATA && d->data_location != DMRG_DEVICE_DATA) {
    set_error("data_location must be DMRG_HOST_DATA or DMRG_DEVICE_DATA");
    return DMRG_ERR_INVALID_ARG;
  }
  p->dimL.assign(d->dimL, d->dimL + d->nL);
  p->dimR.assign(d->dimR, d->dimR + d->nR);
  for (auto v : p->dimL)
    if (v < 0) { set_error("negative left sector dimension"); return DMRG_ERR_INVALID_ARG; }
  for (auto v : p->dimR)
    if (v < 0) { set_error("negative right sector dimension"); return DMRG_ERR_INVALID_ARG; }
  DMRG_TRY(set_pairs(p, d->npairs, d->pair_i, d->pair_k));
  p->terms.assign(d->terms, d->terms + d->nterms);
  for (auto& t : p->terms) {
    if ((t.a_op != DMRG_IDENTITY_OP && (t.a_op < 0 || t.a_op >= d->nopsL)) ||
        (t.b_op != DMRG_IDENTITY_OP && (t.b_op < 0 || t.b_op >= d->nopsR))) {
      set_error("term names a missing operator");
      return DMRG_ERR_INVALID_ARG;
    }
  }
  size_t total = 0;
  DMRG_TRY(layout_ops(d->nopsL, d->opsL, p->dimL, p->opsL, &total));
  DMRG_TRY(layout_ops(d->nopsR, d->opsR, p->dimR, p->opsR, &total));
  p->arena_elems = total;
  p->arena_host.assign(total, 0.0);
  DMRG_TRY(copy_ops(d->nopsL, d->opsL, p->opsL, d->data_location, p));
  DMRG_TRY(copy_ops(d->nopsR, d->opsR, p->opsR, d->data_location, p));
  return DMRG_OK;
}

// The l-1-1-r form (Sec. 4.2, Eq. 12) presented to the record engine: the block-l sector i
// and the two site states form one "left" sector (i, s1, s2) of dimension dim_l(i); the
// factors of block l and r keep their own blocks, and the site factors -- single elements,
// every site state being a sector of its own -- become coefficients of the records
// (stages 2 and 3 of Algorithm 2 are scalar multiplications).  p->opsL holds the block-l
// operators with block-l sector indices; p->terms one entry per term of Eq. 12 (its block-l
// and block-r factors).
dmrg_status validate_and_copy_l11r(const dmrg_l11r_desc* d, dmrg_plan* p,
                                   std::vector<int64_t>* diml) {
  if (!d) {
    set_error("desc is NULL");
    return DMRG_ERR_INVALID_ARG;
  }
  if (d->nl <= 0 || d->nr <= 0 || d->q <= 0 || d->q > 64 || d->nsegs < 0 || d->nterms < 0 ||
      d->nopsl < 0 || d->nopsr < 0 || d->nsops < 0) {
    set_error("bad sector, site, segment, term or operator counts");
    return DMRG_ERR_INVALID_ARG;
  }
  if (!d->diml || !d->dimr || (d->nsegs && (!d->seg_l || !d->seg_s1 || !d->seg_s2 || !d->seg_r)) ||
      (d->nterms && !d->terms) || (d->nopsl && !d->opsl) || (d->nopsr && !d->opsr) ||
      (d->nsops && !d->sops)) {
    set_error("NULL array in desc");
    return DMRG_ERR_INVALID_ARG;
  }
  if (d->data_location != DMRG_HOST_DATA && d->data_location != DMRG_DEVICE_DATA) {
    set_error("data_location must be DMRG_HOST_DATA or DMRG_DEVICE_DATA");
    return DMRG_ERR_INVALID_ARG;
  }
  const int q = d->q;
  diml->assign(d->diml, d->diml + d->nl);
  p->dimR.assign(d->dimr, d->dimr + d->nr);
  for (auto v : *diml)
    if (v < 0) { set_error("negative block-l sector dimension"); return DMRG_ERR_INVALID_ARG; }
  for (auto v : p->dimR)
    if (v < 0) { set_error("negative block-r sector dimension"); return DMRG_ERR_INVALID_ARG; }
  p->dimL.assign((size_t)d->nl * q * q, 0);
  for (int i = 0; i < d->nl; ++i)
    for (int t = 0; t < q * q; ++t) p->dimL[(size_t)i * q * q + t] = (*diml)[i];
  std::vector<int32_t> pi(d->nsegs), pk(d->nsegs);
  for (int g = 0; g < d->nsegs; ++g) {
    const int i = d->seg_l[g], s1 = d->seg_s1[g], s2 = d->seg_s2[g];
    if (i < 0 || i >= d->nl || s1 < 0 || s1 >= q || s2 < 0 || s2 >= q) {
      set_error("segment %d = (%d,%d,%d,%d) out of range", g, i, s1, s2, d->seg_r[g]);
      return DMRG_ERR_INVALID_ARG;
    }
    pi[g] = (i * q + s1) * q + s2;
    pk[g] = d->seg_r[g];
  }
  DMRG_TRY(set_pairs(p, d->nsegs, pi.data(), pk.data()));
  p->terms.clear();
  for (int t = 0; t < d->nterms; ++t) {
    const dmrg_term4& tm = d->terms[t];
    if ((tm.l_op != DMRG_IDENTITY_OP && (tm.l_op < 0 || tm.l_op >= d->nopsl)) ||
        (tm.r_op != DMRG_IDENTITY_OP && (tm.r_op < 0 || tm.r_op >= d->nopsr)) ||
        (tm.s1_op != DMRG_IDENTITY_OP && (tm.s1_op < 0 || tm.s1_op >= d->nsops)) ||
        (tm.s2_op != DMRG_IDENTITY_OP && (tm.s2_op < 0 || tm.s2_op >= d->nsops))) {
      set_error("term %d names a missing operator", t);
      return DMRG_ERR_INVALID_ARG;
    }
    p->terms.push_back(dmrg_term{tm.coef, tm.l_op, tm.r_op});
  }
  size_t total = 0;
  DMRG_TRY(layout_ops(d->nopsl, d->opsl, *diml, p->opsL, &total));
  DMRG_TRY(layout_ops(d->nopsr, d->opsr, p->dimR, p->opsR, &total));
  p->arena_elems = total;
  p->arena_host.assign(total, 0.0);
  DMRG_TRY(copy_ops(d->nopsl, d->opsl, p->opsL, d->data_location, p));
  DMRG_TRY(copy_ops(d->nopsr, d->opsr, p->opsR, d->data_location, p));
  return DMRG_OK;
}

struct Builder {
  std::vector<Job64> jobs;
  std::vector<Seg64> segs;
  std::vector<Tile64> tiles1, tiles2;
};

Operand opnd(int space, int64_t off, int64_t rs, int64_t cs) {
  Operand o;
  o.off = off;
  o.rs = rs;
  o.cs = cs;
  o.space = space;
  o.pad_ = 0;
  return o;
}

void add_tiles(std::vector<Tile64>& tiles, int job, int64_t M, int64_t N) {
  for (int64_t m0 = 0; m0 < std::max<int64_t>(M, 1); m0 += kTileM)
    for (int64_t n0 = 0; n0 < std::max<int64_t>(N, 1); n0 += kTileN)
      tiles.push_back(Tile64{job, (int32_t)m0, (int32_t)n0, 0});
}

// A record's multiplication order, FLOPs and intermediate buffer slot (Sec. 7: the
// workload of each record is known once the plan exists).
void finish_record(dmrg_plan* p, Record& r, int64_t* inter) {
  r.inter_off = -1;
  if (r.a_blk >= 0 && r.b_blk >= 0) {
    int64_t cA = 2 * r.dj * r.di * r.dk + 2 * r.dj * r.dk * r.dl;
    int64_t cB = 2 * r.di * r.dk * r.dl + 2 * r.dj * r.di * r.dl;
    r.a_first = cA <= cB ? 1 : 0;
    p->flops += std::min(cA, cB);
    r.inter_off = *inter;
    *inter += round_up(r.a_first ? r.dj * r.dk : r.di * r.dl, 32);
  } else if (r.a_blk >= 0) {
    p->flops += 2 * r.dj * r.di * r.dk;
  } else if (r.b_blk >= 0) {
    p->flops += 2 * r.di * r.dk * r.dl;
  }
  p->records.push_back(r);
}

// LR form (Eq. 11): one record per term and pair of blocks whose input (i, k) and output
// (j, l) segments are in the sector
void build_records_lr(dmrg_plan* p) {
  const int npairs = (int)p->pair_i.size();
  std::map<std::pair<int, int>, int> pidx;
  for (int q = 0; q < npairs; ++q) pidx[{p->pair_i[q], p->pair_k[q]}] = q;
  const int nL = (int)p->dimL.size(), nR = (int)p->dimR.size();
  std::vector<HostBlock> idL(nL), idR(nR);
  for (int i = 0; i < nL; ++i) idL[i] = HostBlock{i, i, p->dimL[i], p->dimL[i], -1};
  for (int k = 0; k < nR; ++k) idR[k] = HostBlock{k, k, p->dimR[k], p->dimR[k], -1};
  p->records.clear();
  p->flops = 0;
  int64_t inter = 0;
  for (int t = 0; t < (int)p->terms.size(); ++t) {
    const dmrg_term& term = p->terms[t];
    const std::vector<HostBlock>& As = term.a_op == DMRG_IDENTITY_OP ? idL : p->opsL[term.a_op];
    const std::vector<HostBlock>& Bs = term.b_op == DMRG_IDENTITY_OP ? idR : p->opsR[term.b_op];
    for (int ai = 0; ai < (int)As.size(); ++ai) {
      for (int bi = 0; bi < (int)Bs.size(); ++bi) {
        const HostBlock& A = As[ai];
        const HostBlock& B = Bs[bi];
        auto in = pidx.find({A.idx_in, B.idx_in});
        auto out = pidx.find({A.idx_out, B.idx_out});
        if (in == pidx.end() || out == pidx.end()) continue;
        Record r{};
        r.term = t;
        r.a_blk = term.a_op == DMRG_IDENTITY_OP ? -1 : ai;
        r.b_blk = term.b_op == DMRG_IDENTITY_OP ? -1 : bi;
        r.pin = in->second;
        r.pout = out->second;
        r.i = A.idx_in; r.j = A.idx_out; r.k = B.idx_in; r.l = B.idx_out;
        r.di = p->dimL[r.i]; r.dj = p->dimL[r.j]; r.dk = p->dimR[r.k]; r.dl = p->dimR[r.l];
        r.coef = term.coef;
        finish_record(p, r, &inter);
      }
    }
  }
  p->T_elems = (size_t)inter;
}

// l-1-1-r form (Eq. 13 with the blocks of the paragraph after it): one record per term,
// block of l, site elements a[s1' <- s1], b[s2' <- s2] and block of r whose input
// (i, s1, s2, k) and output (j, s1', s2', l) segments are in the sector, with coefficient
// coef * a * b.  Left sectors are the tuples (i * q + s1) * q + s2.
dmrg_status build_records_l11r(dmrg_plan* p, const dmrg_l11r_desc* d,
                               const std::vector<int64_t>& diml) {
  const int q = d->q;
  const int npairs = (int)p->pair_i.size();
  std::map<std::pair<int, int>, int> pidx;
  for (int g = 0; g < npairs; ++g) pidx[{p->pair_i[g], p->pair_k[g]}] = g;
  const int nl = d->nl, nR = (int)p->dimR.size();
  std::vector<HostBlock> idl(nl), idR(nR);
  for (int i = 0; i < nl; ++i) idl[i] = HostBlock{i, i, diml[i], diml[i], -1};
  for (int k = 0; k < nR; ++k) idR[k] = HostBlock{k, k, p->dimR[k], p->dimR[k], -1};
  struct Elem { int in, out; double v; };
  auto site_elems = [&](int o) {
    std::vector<Elem> e;
    if (o == DMRG_IDENTITY_OP) {
      for (int s = 0; s < q; ++s) e.push_back(Elem{s, s, 1.0});
    } else {
      const double* M = d->sops + (size_t)o * q * q;  // row-major [out][in]
      for (int sin = 0; sin < q; ++sin)
        for (int sout = 0; sout < q; ++sout)
          if (M[(size_t)sout * q + sin] != 0.0) e.push_back(Elem{sin, sout, M[(size_t)sout * q + sin]});
    }
    return e;
  };
  p->records.clear();
  p->flops = 0;
  int64_t inter = 0;
  for (int t = 0; t < d->nterms; ++t) {
    const dmrg_term4& tm = d->terms[t];
    const std::vector<HostBlock>& As = tm.l_op == DMRG_IDENTITY_OP ? idl : p->opsL[tm.l_op];
    const std::vector<HostBlock>& Bs = tm.r_op == DMRG_IDENTITY_OP ? idR : p->opsR[tm.r_op];
    const std::vector<Elem> e1 = site_elems(tm.s1_op), e2 = site_elems(tm.s2_op);
    for (int ai = 0; ai < (int)As.size(); ++ai) {
      for (int bi = 0; bi < (int)Bs.size(); ++bi) {
        const HostBlock& A = As[ai];
        const HostBlock& B = Bs[bi];
        for (const Elem& u : e1) {
          for (const Elem& v : e2) {
            const int Iin = (A.idx_in * q + u.in) * q + v.in;
            const int Iout = (A.idx_out * q + u.out) * q + v.out;
            auto in = pidx.find({Iin, B.idx_in});
            auto out = pidx.find({Iout, B.idx_out});
            if (in == pidx.end() || out == pidx.end()) continue;
            Record r{};
            r.term = t;
            r.a_blk = tm.l_op == DMRG_IDENTITY_OP ? -1 : ai;
            r.b_blk = tm.r_op == DMRG_IDENTITY_OP ? -1 : bi;
            r.pin = in->second;
            r.pout = out->second;
            r.i = Iin; r.j = Iout; r.k = B.idx_in; r.l = B.idx_out;
            r.di = diml[A.idx_in]; r.dj = diml[A.idx_out];
            r.dk = p->dimR[r.k]; r.dl = p->dimR[r.l];
            r.coef = tm.coef * u.v * v.v;
            finish_record(p, r, &inter);
          }
        }
      }
    }
  }
  p->T_elems = (size_t)inter;
  return DMRG_OK;
}

// FP64 GEMM work lists from the records: stage-1 intermediates and stage-2 output jobs
dmrg_status build_jobs(dmrg_plan* p, Builder* bld) {
  const int npairs = (int)p->pair_i.size();
  auto A_of = [&](const Record& r) -> const HostBlock& {
    return p->opsL[p->terms[r.term].a_op][r.a_blk];
  };
  auto B_of = [&](const Record& r) -> const HostBlock& {
    return p->opsR[p->terms[r.term].b_op][r.b_blk];
  };

  // stage 1: one job per record with two non-identity factors
  std::vector<std::pair<int64_t, int>> order1;
  for (const Record& r : p->records) {
    if (r.a_blk < 0 || r.b_blk < 0) continue;
    Job64 job{};
    Seg64 s{};
    if (r.a_first) {  // T[dj x dk] = A[dj x di] X[di x dk]
      const HostBlock& A = A_of(r);
      job.C = opnd(SP_T, r.inter_off, r.dk, 1);
      job.M = (int32_t)r.dj;
      job.N = (int32_t)r.dk;
      s.P = opnd(SP_ARENA, A.arena_off, A.cols, 1);
      s.Q = opnd(SP_X, p->pair_off[r.pin], r.dk, 1);
      s.K = (int32_t)r.di;
    } else {          // U[di x dl] = X[di x dk] B^T[dk x dl]
      const HostBlock& B = B_of(r);
      job.C = opnd(SP_T, r.inter_off, r.dl, 1);
      job.M = (int32_t)r.di;
      job.N = (int32_t)r.dl;
      s.P = opnd(SP_X, p->pair_off[r.pin], r.dk, 1);
      s.Q = opnd(SP_ARENA, B.arena_off, 1, B.cols);
      s.K = (int32_t)r.dk;
    }
    s.alpha = 1.0;
    job.axpy = 0.0;
    job.Xaxpy = opnd(SP_X, 0, 0, 0);
    job.seg_begin = (int32_t)bld->segs.size();
    bld->segs.push_back(s);
    job.seg_end = (int32_t)bld->segs.size();
    int jid = (int)bld->jobs.size();
    bld->jobs.push_back(job);
    order1.push_back({(int64_t)s.K, jid});
  }
  // stage 2: one job per output pair
  std::vector<std::vector<int>> by_out(npairs);
  for (int ri = 0; ri < (int)p->records.size(); ++ri) by_out[p->records[ri].pout].push_back(ri);
  std::vector<std::pair<int64_t, int>> order2;
  for (int q = 0; q < npairs; ++q) {
    int i = p->pair_i[q], k = p->pair_k[q];
    Job64 job{};
    job.C = opnd(SP_Y, p->pair_off[q], p->dimR[k], 1);
    job.M = (int32_t)p->dimL[i];
    job.N = (int32_t)p->dimR[k];
    job.axpy = 0.0;
    job.Xaxpy = opnd(SP_X, p->pair_off[q], p->dimR[k], 1);
    job.seg_begin = (int32_t)bld->segs.size();
    int64_t cost = 0;
    for (int ri : by_out[q]) {
      const Record& r = p->records[ri];
      Seg64 s{};
      s.alpha = r.coef;
      if (r.a_blk >= 0 && r.b_blk >= 0) {
        if (r.a_first) {  // Y += coef T[dj x dk] B^T[dk x dl]
          const HostBlock& B = B_of(r);
          s.P = opnd(SP_T, r.inter_off, r.dk, 1);
          s.Q = opnd(SP_ARENA, B.arena_off, 1, B.cols);
          s.K = (int32_t)r.dk;
        } else {          // Y += coef A[dj x di] U[di x dl]
          const HostBlock& A = A_of(r);
          s.P = opnd(SP_ARENA, A.arena_off, A.cols, 1);
          s.Q = opnd(SP_T, r.inter_off, r.dl, 1);
          s.K = (int32_t)r.di;
        }
      } else if (r.a_blk >= 0) {  // (A (x) 1): Y_jl += coef A X_il, k == l
        const HostBlock& A = A_of(r);
        s.P = opnd(SP_ARENA, A.arena_off, A.cols, 1);
        s.Q = opnd(SP_X, p->pair_off[r.pin], r.dk, 1);
        s.K = (int32_t)r.di;
      } else if (r.b_blk >= 0) {  // (1 (x) B): Y_jl += coef X_jk B^T, i == j
        const HostBlock& B = B_of(r);
        s.P = opnd(SP_X, p->pair_off[r.pin], r.dk, 1);
        s.Q = opnd(SP_ARENA, B.arena_off, 1, B.cols);
        s.K = (int32_t)r.dk;
      } else {                    // (1 (x) 1): Y += coef X
        if (r.pin == r.pout) job.axpy += r.coef;  // (other segments: seg_axpy pass)
        continue;
      }
      if (s.K == 0) continue;
      cost += s.K;
      bld->segs.push_back(s);
    }
    job.seg_end = (int32_t)bld->segs.size();
    int jid = (int)bld->jobs.size();
    bld->jobs.push_back(job);
    order2.push_back({cost, jid});
  }
  // longest-first ordering of the tiles of each stage (LPT)
  auto by_cost = [](const std::pair<int64_t, int>& a, const std::pair<int64_t, int>& b) {
    return a.first != b.first ? a.first > b.first : a.second < b.second;
  };
  std::stable_sort(order1.begin(), order1.end(), by_cost);
  std::stable_sort(order2.begin(), order2.end(), by_cost);
  for (auto& pr : order1) add_tiles(bld->tiles1, pr.second, bld->jobs[pr.second].M, bld->jobs[pr.second].N);
  for (auto& pr : order2) {
    const Job64& j = bld->jobs[pr.second];
    if (j.M == 0 || j.N == 0) continue;
    add_tiles(bld->tiles2, pr.second, j.M, j.N);
  }
  return DMRG_OK;
}

template <typename T>
dmrg_status upload(T** dst, const std::vector<T>& src, size_t* bytes, cudaStream_t st) {
  *dst = nullptr;
  if (src.empty()) return DMRG_OK;
  DMRG_CUDA_TRY(cudaMalloc((void**)dst, sizeof(T) * src.size()));
  *bytes += sizeof(T) * src.size();
  DMRG_CUDA_TRY(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(),
                                cudaMemcpyHostToDevice, st));
  return DMRG_OK;
}

// ---------------------------------------------------------------- diagonal of H_SB
// D[off_p + a * dk + b] = sum over the records that map segment p to itself of
// coef * diag(A)[a] * diag(B)[b] (such a record's blocks are diagonal-sector blocks;
// identity factors contribute 1).  In the LR form these are the terms' diagonal blocks; in
// the l-1-1-r form the coefficients carry the diagonal site elements.
struct DiagEntry {
  int64_t a_off, b_off;   // arena offsets of the diagonal blocks, -1 identity
  int64_t a_ld, b_ld;
  double coef;
};

__global__ void diag_kernel(const double* __restrict__ arena, const DiagEntry* __restrict__ ent,
                            const int32_t* __restrict__ ent_beg, const int64_t* __restrict__ pair_off,
                            const int64_t* __restrict__ pair_dk, double* __restrict__ D) {
  const int p = blockIdx.y;
  const int64_t off = pair_off[p], size = pair_off[p + 1] - off, dk = pair_dk[p];
  const int e0 = ent_beg[p], e1 = ent_beg[p + 1];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < size;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / dk, b = e - a * dk;
    double acc = 0.0;
    for (int t = e0; t < e1; ++t) {
      const DiagEntry& d = ent[t];
      const double da = d.a_off == -1 ? 1.0 : arena[d.a_off + a * (d.a_ld + 1)];
      const double db = d.b_off == -1 ? 1.0 : arena[d.b_off + b * (d.b_ld + 1)];
      acc = fma(d.coef * da, db, acc);
    }
    D[off + e] = acc;
  }
}

}  // namespace

namespace dmrg {

dmrg_status compute_diagonal(dmrg_plan* p, double* d, cudaStream_t st) {
  const int npairs = (int)p->pair_i.size();
  if (npairs == 0 || p->n == 0) return DMRG_OK;
  std::vector<std::vector<DiagEntry>> per(npairs);
  for (const Record& r : p->records) {
    if (r.pin != r.pout) continue;
    DiagEntry e{-1, -1, 0, 0, r.coef};
    if (r.a_blk >= 0) {
      const HostBlock& hb = p->opsL[p->terms[r.term].a_op][r.a_blk];
      e.a_off = hb.arena_off;
      e.a_ld = hb.cols;
    }
    if (r.b_blk >= 0) {
      const HostBlock& hb = p->opsR[p->terms[r.term].b_op][r.b_blk];
      e.b_off = hb.arena_off;
      e.b_ld = hb.cols;
    }
    per[r.pin].push_back(e);
  }
  std::vector<DiagEntry> ent;
  std::vector<int32_t> beg(npairs + 1, 0);
  for (int q = 0; q < npairs; ++q) {
    ent.insert(ent.end(), per[q].begin(), per[q].end());
    beg[q + 1] = (int32_t)ent.size();
  }
  if (ent.empty()) ent.push_back(DiagEntry{-1, -1, 0, 0, 0.0});  // (no record: D = 0)
  std::vector<int64_t> dk(npairs);
  for (int q = 0; q < npairs; ++q) dk[q] = p->dimR[p->pair_k[q]];
  DiagEntry* d_ent = nullptr;
  int32_t* d_beg = nullptr;
  int64_t *d_off = nullptr, *d_dk = nullptr;
  size_t dummy = 0;
  DMRG_TRY(upload(&d_ent, ent, &dummy, st));
  DMRG_TRY(upload(&d_beg, beg, &dummy, st));
  DMRG_TRY(upload(&d_off, p->pair_off, &dummy, st));
  DMRG_TRY(upload(&d_dk, dk, &dummy, st));
  dim3 grid(64, npairs);
  diag_kernel<<<grid, 256, 0, st>>>(p->arena, d_ent, d_beg, d_off, d_dk, d);
  note_launch();
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(st);
  cudaFree(d_ent);
  cudaFree(d_beg);
  cudaFree(d_off);
  cudaFree(d_dk);
  if (e != cudaSuccess) {
    set_error("diag_kernel: %s", cudaGetErrorString(e));
    return DMRG_ERR_CUDA;
  }
  return DMRG_OK;
}

template <typename T>
__global__ void seg_axpy_kernel(const SegAxpyGroup* __restrict__ groups,
                                const SegAxpyEntry* __restrict__ ent, const T* __restrict__ x,
                                T* __restrict__ y) {
  const SegAxpyGroup g = groups[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.size;
       e += (int64_t)gridDim.x * blockDim.x) {
    T acc = y[g.dst_off + e];
    for (int t = g.beg; t < g.end; ++t) {
      const SegAxpyEntry en = ent[t];
      if constexpr (sizeof(T) == 8) acc = fma(en.coef, x[en.src_off + e], acc);
      else acc = fmaf((float)en.coef, x[en.src_off + e], acc);
    }
    y[g.dst_off + e] = acc;
  }
}

dmrg_status launch_seg_axpy(const dmrg_plan* p, const double* x, double* y, const float* x32,
                            float* y32, cudaStream_t st) {
  if (p->n_sax_groups == 0) return DMRG_OK;
  const dim3 grid((unsigned)std::min<int64_t>(64, (p->sax_max_size + 255) / 256), (unsigned)p->n_sax_groups);
  if (x32) seg_axpy_kernel<float><<<grid, 256, 0, st>>>(p->d_sax_groups, p->d_sax_entries, x32, y32);
  else seg_axpy_kernel<double><<<grid, 256, 0, st>>>(p->d_sax_groups, p->d_sax_entries, x, y);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

}  // namespace dmrg

namespace {

// a plan with validated options (defaults if opt is NULL)
dmrg_status new_plan(const dmrg_options* opt, dmrg_plan** out) {
  dmrg_plan* p = new (std::nothrow) dmrg_plan();
  if (!p) {
    set_error("host allocation failed");
    return DMRG_ERR_OOM;
  }
  if (opt) p->opt = *opt; else dmrg_options_default(&p->opt);
  if (p->opt.max_subspace < 2 || p->opt.max_subspace > DMRG_MAX_SUBSPACE ||
      p->opt.max_iter < 1 || !(p->opt.tol >= 0.0) ||
      (int)p->opt.prec < 0 || (int)p->opt.prec > 4 ||
      (p->opt.anchor_prec != DMRG_PREC_FP64 && p->opt.anchor_prec != DMRG_PREC_FP64_TC) ||
      p->opt.vector_arith < DMRG_VEC_FP64 || p->opt.vector_arith > DMRG_VEC_SPLIT ||
      (p->opt.autotune != 0 && p->opt.autotune != 1) ||
      (p->opt.graphs != 0 && p->opt.graphs != 1) ||
      (p->opt.restart_keep != 1 && p->opt.restart_keep != 2)) {
    set_error("options out of range (max_subspace must be in [2, %d])", DMRG_MAX_SUBSPACE);
    delete p;
    return DMRG_ERR_INVALID_ARG;
  }
  *out = p;
  return DMRG_OK;
}

// FP64 work lists, device arena, intermediates and the diagonal of a plan whose records
// exist; on failure the plan is destroyed
dmrg_status finish_plan(dmrg_plan* p, cudaStream_t st, dmrg_plan** out) {
  cudaGetDevice(&p->device);
  Builder bld;
  dmrg_status s = build_jobs(p, &bld);
  if (s != DMRG_OK) { delete p; return s; }
  auto fail = [&](dmrg_status st_) { dmrg_plan_destroy(p); return st_; };
  if (p->arena_elems) {
    if (cudaMalloc((void**)&p->arena, sizeof(double) * p->arena_elems) != cudaSuccess) {
      set_error("cudaMalloc of %zu bytes for the operator arena failed",
                sizeof(double) * p->arena_elems);
      return fail(DMRG_ERR_OOM);
    }
    p->device_bytes += sizeof(double) * p->arena_elems;
    if (cudaMemcpyAsync(p->arena, p->arena_host.data(), sizeof(double) * p->arena_elems,
                        cudaMemcpyHostToDevice, st) != cudaSuccess) {
      set_error("arena upload failed");
      return fail(DMRG_ERR_CUDA);
    }
  }
  if (p->T_elems) {
    if (cudaMalloc((void**)&p->T, sizeof(double) * p->T_elems) != cudaSuccess) {
      set_error("cudaMalloc for the intermediates failed");
      return fail(DMRG_ERR_OOM);
    }
    p->device_bytes += sizeof(double) * p->T_elems;
  }
  if ((s = upload(&p->d_jobs, bld.jobs, &p->device_bytes, st)) != DMRG_OK) return fail(s);
  if ((s = upload(&p->d_segs, bld.segs, &p->device_bytes, st)) != DMRG_OK) return fail(s);
  if ((s = upload(&p->d_tiles1, bld.tiles1, &p->device_bytes, st)) != DMRG_OK) return fail(s);
  if ((s = upload(&p->d_tiles2, bld.tiles2, &p->device_bytes, st)) != DMRG_OK) return fail(s);
  p->ntiles1 = (int64_t)bld.tiles1.size();
  p->ntiles2 = (int64_t)bld.tiles2.size();
  {
    // cross-segment identity terms, grouped by output segment in record order
    std::map<int, std::vector<SegAxpyEntry>> by_dst;
    for (const Record& r : p->records)
      if (r.a_blk < 0 && r.b_blk < 0 && r.pin != r.pout && r.coef != 0.0)
        by_dst[r.pout].push_back(SegAxpyEntry{p->pair_off[r.pin], r.coef});
    std::vector<SegAxpyGroup> groups;
    std::vector<SegAxpyEntry> ent;
    for (auto& kv : by_dst) {
      const int64_t size = p->pair_off[kv.first + 1] - p->pair_off[kv.first];
      groups.push_back(SegAxpyGroup{p->pair_off[kv.first], size, (int32_t)ent.size(),
                                    (int32_t)(ent.size() + kv.second.size())});
      ent.insert(ent.end(), kv.second.begin(), kv.second.end());
      p->sax_max_size = std::max(p->sax_max_size, size);
    }
    if ((s = upload(&p->d_sax_groups, groups, &p->device_bytes, st)) != DMRG_OK) return fail(s);
    if ((s = upload(&p->d_sax_entries, ent, &p->device_bytes, st)) != DMRG_OK) return fail(s);
    p->n_sax_groups = (int32_t)groups.size();
  }
  if (p->n > 0) {
    if (cudaMalloc((void**)&p->D, sizeof(double) * p->n) != cudaSuccess) {
      set_error("cudaMalloc for the diagonal failed");
      return fail(DMRG_ERR_OOM);
    }
    p->device_bytes += sizeof(double) * p->n;
    if ((s = compute_diagonal(p, p->D, st)) != DMRG_OK) return fail(s);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("plan upload: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(DMRG_ERR_CUDA);
  }
  *out = p;
  return DMRG_OK;
}

}  // namespace

extern "C" {

dmrg_status dmrg_plan_create(const dmrg_superblock_desc* desc, const dmrg_options* opt,
                             void* stream, dmrg_plan** out) {
  if (!out) {
    set_error("out is NULL");
    return DMRG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  dmrg_plan* p = nullptr;
  DMRG_TRY(new_plan(opt, &p));
  cudaStream_t st = (cudaStream_t)stream;
  dmrg_status s = validate_and_copy(desc, p);
  if (s != DMRG_OK) { delete p; return s; }
  build_records_lr(p);
  return finish_plan(p, st, out);
}

dmrg_status dmrg_plan_create_l11r(const dmrg_l11r_desc* desc, const dmrg_options* opt,
                                  void* stream, dmrg_plan** out) {
  if (!out) {
    set_error("out is NULL");
    return DMRG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  dmrg_plan* p = nullptr;
  DMRG_TRY(new_plan(opt, &p));
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> diml;
  dmrg_status s = validate_and_copy_l11r(desc, p, &diml);
  if (s == DMRG_OK) s = build_records_l11r(p, desc, diml);
  if (s != DMRG_OK) { delete p; return s; }
  return finish_plan(p, st, out);
}

void dmrg_plan_destroy(dmrg_plan* p) {
  if (!p) return;
  dmrg_plan_trim(p);
  destroy_tc(p);
  destroy_oz(p);
  cudaFree(p->arena);
  cudaFree(p->T);
  cudaFree(p->D);
  cudaFree(p->d_jobs);
  cudaFree(p->d_segs);
  cudaFree(p->d_tiles1);
  cudaFree(p->d_tiles2);
  cudaFree(p->d_sax_groups);
  cudaFree(p->d_sax_entries);
  delete p;
}

dmrg_status dmrg_plan_get_stats(const dmrg_plan* p, dmrg_plan_stats* s) {
  if (!p || !s) {
    set_error("NULL argument");
    return DMRG_ERR_INVALID_ARG;
  }
  s->n = p->n;
  s->records = (int64_t)p->records.size();
  s->flops = p->flops;
  s->tiles_stage1 = p->ntiles1;
  s->tiles_stage2 = p->ntiles2;
  s->device_bytes = (int64_t)p->device_bytes;
  tc_schedule_stats(p, s->tc_schedule, s->tc_tune_us);
  return DMRG_OK;
}

dmrg_status dmrg_plan_autotune(dmrg_plan* p, dmrg_precision prec, void* stream) {
  if (!p) {
    set_error("NULL plan");
    return DMRG_ERR_INVALID_ARG;
  }
  if (!tc_lowprec(prec)) {
    set_error("autotune: precision must be DMRG_PREC_TF32, DMRG_PREC_BF16X3 or DMRG_PREC_BF16X2");
    return DMRG_ERR_INVALID_ARG;
  }
  if (p->n == 0) return DMRG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  DMRG_TRY(tune_project_tc(p, prec, st));
  DMRG_CUDA_TRY(cudaStreamSynchronize(st));
  return DMRG_OK;
}

dmrg_status dmrg_plan_set_tile_schedule(dmrg_plan* p, dmrg_precision prec, int32_t stage1,
                                        int32_t stage2, void* stream) {
  if (!p) {
    set_error("NULL plan");
    return DMRG_ERR_INVALID_ARG;
  }
  if (!tc_lowprec(prec)) {
    set_error("tile schedule: precision must be DMRG_PREC_TF32, DMRG_PREC_BF16X3 or DMRG_PREC_BF16X2");
    return DMRG_ERR_INVALID_ARG;
  }
  if (p->n == 0) return DMRG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  DMRG_TRY(set_schedule_tc(p, prec, stage1, stage2, st));
  DMRG_CUDA_TRY(cudaStreamSynchronize(st));
  return DMRG_OK;
}

dmrg_status dmrg_diagonal(dmrg_plan* p, double* d, void* stream) {
  if (!p || (!d && p->n)) {
    set_error("NULL argument");
    return DMRG_ERR_INVALID_ARG;
  }
  if (p->n == 0) return DMRG_OK;
  DMRG_CUDA_TRY(cudaMemcpyAsync(d, p->D, sizeof(double) * p->n, cudaMemcpyDeviceToDevice,
                                (cudaStream_t)stream));
  return DMRG_OK;
}

dmrg_status dmrg_project_prec(dmrg_plan* p, dmrg_precision prec, const double* x, double* y,
                              void* stream) {
  if (!p || (p->n && (!x || !y))) {
    set_error("NULL argument");
    return DMRG_ERR_INVALID_ARG;
  }
  if (p->n == 0) return DMRG_OK;
  if ((const double*)y < x + p->n && x < (const double*)y + p->n) {
    set_error("x and y overlap");
    return DMRG_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == DMRG_PREC_FP64) return launch_project_fp64(p, x, y, st);
  if (prec == DMRG_PREC_FP64_TC) return launch_project_oz(p, x, y, st);
  if (tc_lowprec(prec)) return launch_project_tc(p, prec, x, y, st);
  set_error("unknown precision %d", (int)prec);
  return DMRG_ERR_INVALID_ARG;
}

dmrg_status dmrg_project(dmrg_plan* p, const double* x, double* y, void* stream) {
  return dmrg_project_prec(p, DMRG_PREC_FP64, x, y, stream);
}

dmrg_status dmrg_project_digits(dmrg_plan* p, int32_t digits, const double* x, double* y,
                                void* stream) {
  if (!p || (p->n && (!x || !y)) || digits < 2 || digits > 7) {
    set_error("dmrg_project_digits: NULL argument or digits outside [2, 7]");
    return DMRG_ERR_INVALID_ARG;
  }
  if (p->n == 0) return DMRG_OK;
  if ((const double*)y < x + p->n && x < (const double*)y + p->n) {
    set_error("x and y overlap");
    return DMRG_ERR_INVALID_ARG;
  }
  return launch_project_oz(p, x, y, (cudaStream_t)stream, digits);
}

}  // extern "C"
