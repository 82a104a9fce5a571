// Plan construction for formatted H-matrix operations (see acr_plan.h).
#include "acr_plan.h"

#include <algorithm>
#include <cstdio>
#include <stdexcept>
#include <unordered_map>

namespace acr {

namespace {

constexpr int TILE = 64;    // output tile (rows and columns) of the grouped GEMM

enum { TERM_A = 0, TERM_B = 1, TERM_D = 2 };

struct Term {
  int prod, t, r, s, type, anode, bnode, a_role, b_role, coef;
  int64_t off;   // scratch offset of the computed factor (W, Y or the dense product)
  int ld;        // its leading dimension
};

struct Dim { int32_t st, rb, ri; };
inline Dim dconst(int v) { return Dim{v, -1, 0}; }
inline Dim drank(int rb, int ri) { return Dim{0, rb, ri}; }

struct Builder {
  const Structure& S;
  const OpDesc& op;
  const PlanParams& pp;
  Plan& P;
  int nroles;
  int kc;
  std::vector<Term> terms;
  std::unordered_map<int64_t, std::vector<int>> terms_at;   // key t*ncl+s

  Builder(const Structure& s_, const OpDesc& o, const PlanParams& p, Plan& pl)
      : S(s_), op(o), pp(p), P(pl), nroles(o.nroles), kc(p.kc) {}

  int bdense(int role) const { return 3 * role; }
  int bU(int role) const { return 3 * role + 1; }
  int bV(int role) const { return 3 * role + 2; }
  int bscr() const { return 3 * nroles; }
  int rscr() const { return nroles; }
  int64_t key(int t, int s) const { return (int64_t)t * (int64_t)S.cl.size() + s; }

  int64_t alloc(int64_t n) {
    int64_t o = P.scratch;
    P.scratch += (n + 3) & ~int64_t(3);
    return o;
  }
  int alloc_rank() { return P.scratch_ranks++; }

  int begin_group(int cbuf, int64_t coff, int ldc, Dim m, Dim n, int beta) {
    GGroup g;
    g.coff = coff; g.cbuf = cbuf; g.ldc = ldc;
    g.m_st = m.st; g.m_rb = m.rb; g.m_ri = m.ri;
    g.n_st = n.st; g.n_rb = n.rb; g.n_ri = n.ri;
    g.ib = g.ie = (int)P.items.size();
    g.beta = beta; g.pad = 0;
    P.groups.push_back(g);
    return (int)P.groups.size() - 1;
  }
  void add_item(int abuf, int64_t aoff, int lda, int aflags, int bbuf, int64_t boff, int ldb,
                int bflags, Dim k, Dim rows, int row_off, int coef, int seed = 0, int orow0 = 0,
                int guard0 = -1, int guard1 = -1) {
    GItem it;
    it.aoff = aoff; it.boff = boff; it.abuf = abuf; it.bbuf = bbuf; it.lda = lda; it.ldb = ldb;
    it.aflags = aflags; it.bflags = bflags;
    it.k_st = k.st; it.k_rb = k.rb; it.k_ri = k.ri;
    it.r_st = rows.st; it.r_rb = rows.rb; it.r_ri = rows.ri;
    it.row_off = row_off; it.coef = coef; it.seed = seed; it.omega_row0 = orow0;
    it.guard0 = guard0; it.guard1 = guard1;
    P.items.push_back(it);
    P.groups.back().ie = (int)P.items.size();
  }
  void stage(int kind, int beg, int end, int tag = -1) {
    if (end > beg) P.stages.push_back(Stage{kind, beg, end, tag});
  }

  // ---------------------------------------------------------------- terms
  void mm(int prod, int t, int r, int s) {
    const OpDesc::Prod& pr = op.prods[prod];
    int a = S.node(t, r), b = S.node(r, s);
    if (a < 0 || b < 0) throw std::runtime_error("product operand outside the block tree");
    int ka = S.bn[a].kind, kb = S.bn[b].kind;
    if (ka == BK_INNER && kb == BK_INNER) {
      const Cluster &ct = S.cl[t], &cr = S.cl[r], &cs = S.cl[s];
      for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 2; ++k)
          for (int j = 0; j < 2; ++j) mm(prod, ct.child[i], cr.child[k], cs.child[j]);
      return;
    }
    Term q;
    q.prod = prod; q.t = t; q.r = r; q.s = s; q.anode = a; q.bnode = b;
    q.a_role = pr.a_role; q.b_role = pr.b_role; q.coef = pr.coef; q.off = -1; q.ld = 0;
    if (ka == BK_LOWRANK) q.type = TERM_A;
    else if (kb == BK_LOWRANK) q.type = TERM_B;
    else if (ka == BK_DENSE && kb == BK_DENSE) q.type = TERM_D;
    else throw std::runtime_error("unbalanced block trees (dense x inner) are not supported");
    terms_at[key(t, s)].push_back((int)terms.size());
    terms.push_back(q);
  }

  // ---------------------------------------------------------------- phase 1
  void phase1() {
    const int lsz = S.lsz;
    std::vector<int> leaves;
    // stage 1a: small inner products M
    int g0 = (int)P.groups.size();
    struct MRef { int term, leaf_node; int64_t off; };
    std::vector<MRef> mrefs;
    for (int qi = 0; qi < (int)terms.size(); ++qi) {
      Term& q = terms[qi];
      if (q.type == TERM_A) {
        q.ld = S.cl[q.s].size;
        q.off = alloc((int64_t)q.ld * kc);
        int la = S.bn[q.anode].leaf;
        leaves.clear();
        S.subtree_leaves(q.bnode, leaves);
        const Cluster& cr = S.cl[q.r];
        for (int bnode : leaves) {
          if (S.bn[bnode].kind != BK_LOWRANK) continue;
          int lb = S.bn[bnode].leaf;
          const Cluster& crb = S.cl[S.bn[bnode].t];
          int64_t moff = alloc((int64_t)kc * kc);
          mrefs.push_back(MRef{qi, bnode, moff});
          // M = U_b^T V_a[r_b]   (k_b x k_a)
          begin_group(bscr(), moff, kc, drank(q.b_role, lb), drank(q.a_role, la), -1);
          add_item(bU(q.b_role), S.lr_row0[lb] * kc, crb.size, FL_T,
                   bV(q.a_role), S.lr_col0[la] * kc + (crb.begin - cr.begin), cr.size, 0,
                   dconst(crb.size), drank(q.b_role, lb), 0, 0);
        }
      } else if (q.type == TERM_B) {
        q.ld = S.cl[q.t].size;
        q.off = alloc((int64_t)q.ld * kc);
        int lb = S.bn[q.bnode].leaf;
        leaves.clear();
        S.subtree_leaves(q.anode, leaves);
        const Cluster& cr = S.cl[q.r];
        for (int anode : leaves) {
          if (S.bn[anode].kind != BK_LOWRANK) continue;
          int la = S.bn[anode].leaf;
          const Cluster& cra = S.cl[S.bn[anode].s];
          int64_t moff = alloc((int64_t)kc * kc);
          mrefs.push_back(MRef{qi, anode, moff});
          // M' = V_a^T U_b[r_a]   (k_a x k_b)
          begin_group(bscr(), moff, kc, drank(q.a_role, la), drank(q.b_role, lb), -1);
          add_item(bV(q.a_role), S.lr_col0[la] * kc, cra.size, FL_T,
                   bU(q.b_role), S.lr_row0[lb] * kc + (cra.begin - cr.begin), cr.size, 0,
                   dconst(cra.size), drank(q.a_role, la), 0, 0);
        }
      }
    }
    stage(ST_GEMM, g0, (int)P.groups.size(), TAG_M);
    // index M by (term, leaf node)
    std::unordered_map<int64_t, int64_t> moff_of;
    for (const MRef& m : mrefs) moff_of[(int64_t)m.term * (int64_t)S.bn.size() + m.leaf_node] = m.off;

    // stage 1b: chunked factors W = B^T V_a, Y = A U_b, dense products
    g0 = (int)P.groups.size();
    for (int qi = 0; qi < (int)terms.size(); ++qi) {
      Term& q = terms[qi];
      if (q.type == TERM_A) {
        int la = S.bn[q.anode].leaf;
        const Cluster& cr = S.cl[q.r];
        const Cluster& cs = S.cl[q.s];
        leaves.clear();
        S.subtree_leaves(q.bnode, leaves);
        for (int c0 = cs.begin; c0 < cs.begin + cs.size; c0 += lsz) {
          begin_group(bscr(), q.off + (c0 - cs.begin), q.ld, dconst(lsz), drank(q.a_role, la), -1);
          for (int bnode : leaves) {
            const BNode& b = S.bn[bnode];
            const Cluster& crb = S.cl[b.t];
            const Cluster& csb = S.cl[b.s];
            if (c0 < csb.begin || c0 >= csb.begin + csb.size) continue;
            if (b.kind == BK_DENSE) {
              // W[c] += B_b^T V_a[r_b]
              add_item(bdense(q.b_role), S.dense_off(b.leaf), lsz, FL_T,
                       bV(q.a_role), S.lr_col0[la] * kc + (crb.begin - cr.begin), cr.size, 0,
                       dconst(lsz), dconst(lsz), 0, 0);
              P.flops_static += 2LL * lsz * lsz * kc;
            } else {
              // W[c] += V_b[c] M
              int64_t moff = moff_of.at((int64_t)qi * (int64_t)S.bn.size() + bnode);
              add_item(bV(q.b_role), S.lr_col0[b.leaf] * kc + (c0 - csb.begin), csb.size, 0,
                       bscr(), moff, kc, 0, drank(q.b_role, b.leaf), dconst(lsz), 0, 0);
            }
          }
        }
      } else if (q.type == TERM_B) {
        int lb = S.bn[q.bnode].leaf;
        const Cluster& cr = S.cl[q.r];
        const Cluster& ct = S.cl[q.t];
        leaves.clear();
        S.subtree_leaves(q.anode, leaves);
        for (int c0 = ct.begin; c0 < ct.begin + ct.size; c0 += lsz) {
          begin_group(bscr(), q.off + (c0 - ct.begin), q.ld, dconst(lsz), drank(q.b_role, lb), -1);
          for (int anode : leaves) {
            const BNode& a = S.bn[anode];
            const Cluster& cta = S.cl[a.t];
            const Cluster& csa = S.cl[a.s];
            if (c0 < cta.begin || c0 >= cta.begin + cta.size) continue;
            if (a.kind == BK_DENSE) {
              // Y[c] += A_a U_b[r_a]
              add_item(bdense(q.a_role), S.dense_off(a.leaf), lsz, 0,
                       bU(q.b_role), S.lr_row0[lb] * kc + (csa.begin - cr.begin), cr.size, 0,
                       dconst(lsz), dconst(lsz), 0, 0);
              P.flops_static += 2LL * lsz * lsz * kc;
            } else {
              int64_t moff = moff_of.at((int64_t)qi * (int64_t)S.bn.size() + anode);
              add_item(bU(q.a_role), S.lr_row0[a.leaf] * kc + (c0 - cta.begin), cta.size, 0,
                       bscr(), moff, kc, 0, drank(q.a_role, a.leaf), dconst(lsz), 0, 0);
            }
          }
        }
      } else {
        // dense x dense: materialise only if the target is not a dense leaf of C
        int cn = S.node(q.t, q.s);
        if (cn >= 0 && S.bn[cn].kind == BK_DENSE) continue;
        q.ld = lsz;
        q.off = alloc((int64_t)lsz * lsz);
        begin_group(bscr(), q.off, lsz, dconst(lsz), dconst(lsz), -1);
        add_item(bdense(q.a_role), S.dense_off(S.bn[q.anode].leaf), lsz, 0,
                 bdense(q.b_role), S.dense_off(S.bn[q.bnode].leaf), lsz, 0,
                 dconst(lsz), dconst(lsz), 0, 0);
        P.flops_static += 2LL * lsz * lsz * lsz;
      }
    }
    stage(ST_GEMM, g0, (int)P.groups.size(), TAG_FACT);
  }

  // ---------------------------------------------------------------- phase 2
  struct LItem {
    bool dense;            // X = dense product (lsz x lsz), Z = identity
    int xbuf; int64_t xoff; int xld; int xrows; int row_off;
    int zbuf; int64_t zoff; int zld; int zrows; int col_off;
    Dim k; int cap; int coef;
    int g0 = -1, g1 = -1;  // operand buffers a dense product depends on
    int64_t sp_off;        // scratch for S_i (k x p) then P_i (k x r)
  };

  // terms restricted / embedded into target leaf (tc, sc)
  void collect_terms(int tc, int sc, bool lowrank, std::vector<int>& anc_self,
                     std::vector<int>& desc) {
    const BNode& root = S.bn[op.c_node];
    int t = tc, s = sc;
    while (true) {
      auto it = terms_at.find(key(t, s));
      if (it != terms_at.end())
        for (int q : it->second) anc_self.push_back(q);
      if (t == root.t && s == root.s) break;
      t = S.cl[t].parent;
      s = S.cl[s].parent;
      if (t < 0 || s < 0) break;
    }
    if (!lowrank) return;
    std::vector<std::pair<int, int>> st;
    const Cluster &ct = S.cl[tc], &cs = S.cl[sc];
    if (ct.child[0] >= 0 && cs.child[0] >= 0)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) st.push_back({ct.child[i], cs.child[j]});
    while (!st.empty()) {
      auto [a, b] = st.back();
      st.pop_back();
      auto it = terms_at.find(key(a, b));
      if (it != terms_at.end())
        for (int q : it->second) desc.push_back(q);
      const Cluster &ca = S.cl[a], &cb = S.cl[b];
      if (ca.child[0] >= 0 && cb.child[0] >= 0)
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j) st.push_back({ca.child[i], cb.child[j]});
    }
  }

  // restricted (ancestor or self) term as an item on target rows tc, cols sc
  LItem term_item(const Term& q, int tc, int sc, bool embedded) {
    LItem li{};
    const Cluster &ct = S.cl[q.t], &cs = S.cl[q.s];
    const Cluster &ctc = S.cl[tc], &csc = S.cl[sc];
    int rdelta = embedded ? 0 : ctc.begin - ct.begin;   // rows of the term taken
    int cdelta = embedded ? 0 : csc.begin - cs.begin;
    li.xrows = embedded ? ct.size : ctc.size;
    li.zrows = embedded ? cs.size : csc.size;
    li.row_off = embedded ? ct.begin - ctc.begin : 0;
    li.col_off = embedded ? cs.begin - csc.begin : 0;
    li.coef = q.coef;
    li.dense = false;
    if (q.type == TERM_A) {
      int la = S.bn[q.anode].leaf;
      li.xbuf = bU(q.a_role); li.xoff = S.lr_row0[la] * kc + rdelta; li.xld = ct.size;
      li.zbuf = bscr(); li.zoff = q.off + cdelta; li.zld = q.ld;
      li.k = drank(q.a_role, la); li.cap = kc;
    } else if (q.type == TERM_B) {
      int lb = S.bn[q.bnode].leaf;
      li.xbuf = bscr(); li.xoff = q.off + rdelta; li.xld = q.ld;
      li.zbuf = bV(q.b_role); li.zoff = S.lr_col0[lb] * kc + cdelta; li.zld = cs.size;
      li.k = drank(q.b_role, lb); li.cap = kc;
    } else {
      li.dense = true;
      li.xbuf = bscr(); li.xoff = q.off; li.xld = S.lsz;
      li.zbuf = -1; li.zoff = 0; li.zld = 0;
      li.k = dconst(S.lsz); li.cap = S.lsz;
      li.xrows = S.lsz; li.zrows = S.lsz;
      li.g0 = bdense(q.a_role); li.g1 = bdense(q.b_role);
    }
    return li;
  }

  void phase2() {
    const int lsz = S.lsz;
    std::vector<int> tleaves;
    S.subtree_leaves(op.c_node, tleaves);
    const int cr = op.c_role;

    // ---- dense targets, and the per-target item lists of low-rank ones
    int gdense0 = (int)P.groups.size();
    struct LT { int node; std::vector<LItem> items; int p; int64_t y, q, bt; TInfo ti; };
    std::vector<LT> lts;
    std::vector<int> anc, desc;
    for (int node : tleaves) {
      const BNode& c = S.bn[node];
      anc.clear(); desc.clear();
      bool lowrank = c.kind == BK_LOWRANK;
      collect_terms(c.t, c.s, lowrank, anc, desc);
      const Cluster &ct = S.cl[c.t], &cs = S.cl[c.s];
      if (!lowrank) {
        ++P.n_dense_targets;
        begin_group(bdense(cr), S.dense_off(c.leaf), lsz, dconst(lsz), dconst(lsz), op.alpha);
        for (const auto& ad : op.adds)
          add_item(bdense(ad.m_role), S.dense_off(c.leaf), lsz, 0, -1, 0, 0, FL_IDENT,
                   dconst(lsz), dconst(lsz), 0, ad.coef);
        for (int qi : anc) {
          const Term& q = terms[qi];
          if (q.type == TERM_D) {
            add_item(bdense(q.a_role), S.dense_off(S.bn[q.anode].leaf), lsz, 0,
                     bdense(q.b_role), S.dense_off(S.bn[q.bnode].leaf), lsz, 0,
                     dconst(lsz), dconst(lsz), 0, q.coef);
            P.flops_static += 2LL * lsz * lsz * lsz;
          } else {
            LItem li = term_item(q, c.t, c.s, false);
            add_item(li.xbuf, li.xoff, li.xld, 0, li.zbuf, li.zoff, li.zld, FL_T,
                     li.k, dconst(lsz), 0, li.coef);
          }
        }
        continue;
      }
      ++P.n_lr_targets;
      LT lt;
      lt.node = node;
      int lc = c.leaf;
      if (op.alpha >= 0) {
        LItem li{};
        li.dense = false;
        li.xbuf = bU(cr); li.xoff = S.lr_row0[lc] * kc; li.xld = ct.size; li.xrows = ct.size;
        li.zbuf = bV(cr); li.zoff = S.lr_col0[lc] * kc; li.zld = cs.size; li.zrows = cs.size;
        li.row_off = li.col_off = 0; li.k = drank(cr, lc); li.cap = kc; li.coef = op.alpha;
        lt.items.push_back(li);
      }
      for (const auto& ad : op.adds) {
        LItem li{};
        li.dense = false;
        li.xbuf = bU(ad.m_role); li.xoff = S.lr_row0[lc] * kc; li.xld = ct.size; li.xrows = ct.size;
        li.zbuf = bV(ad.m_role); li.zoff = S.lr_col0[lc] * kc; li.zld = cs.size; li.zrows = cs.size;
        li.row_off = li.col_off = 0; li.k = drank(ad.m_role, lc); li.cap = kc; li.coef = ad.coef;
        lt.items.push_back(li);
      }
      for (int qi : anc) {
        const Term& q = terms[qi];
        if (q.type == TERM_D) {   // a dense product at this (bottom) low-rank leaf
          LItem li = term_item(q, c.t, c.s, true);
          lt.items.push_back(li);
        } else {
          lt.items.push_back(term_item(q, c.t, c.s, false));
        }
      }
      for (int qi : desc) lt.items.push_back(term_item(terms[qi], c.t, c.s, true));
      lts.push_back(std::move(lt));
    }

    // ---- scratch for low-rank targets
    int64_t capsum_max = 0;
    for (LT& lt : lts) {
      const BNode& c = S.bn[lt.node];
      int m = S.cl[c.t].size, n = S.cl[c.s].size;
      int64_t capsum = 0;
      for (const LItem& li : lt.items) capsum += li.cap;
      capsum_max = std::max(capsum_max, capsum);
      int p = (int)std::min<int64_t>(std::min(kc + pp.oversample, TILE), std::max<int64_t>(capsum, 1));
      lt.p = p;
      lt.y = alloc((int64_t)m * p);
      lt.q = alloc((int64_t)m * p);
      lt.bt = alloc((int64_t)n * p);
      for (LItem& li : lt.items) li.sp_off = alloc((int64_t)li.cap * p);
      TInfo& ti = lt.ti;
      ti.g_off = alloc((int64_t)pp.gram_scale * p * p);
      ti.t_off = alloc((int64_t)p * p);
      ti.h_off = alloc((int64_t)pp.gram_scale * p * p);
      ti.w_off = alloc((int64_t)p * p);
      ti.p = p; ti.m = m; ti.n = n;
      ti.r_ri = alloc_rank();
      ti.c_leaf = c.leaf;
      ti.seed = 0;
      ti.sk_beg = (int)P.stack.size();
      for (const LItem& li : lt.items) {
        if (li.dense)
          P.stack.push_back(StackDim{lsz, -1, 0, li.g0, li.g1});
        else
          P.stack.push_back(StackDim{li.k.st, li.k.rb, li.k.ri, li.xbuf, li.zbuf});
      }
      ti.sk_end = (int)P.stack.size();
      P.targets.push_back(ti);
    }
    for (size_t i = 0; i < lts.size(); ++i) P.targets[i].seed = (int)(1000003u * (uint32_t)(lts[i].node + 1));

    stage(ST_GEMM, gdense0, (int)P.groups.size(), TAG_DENSE);
    // S_i = Z_i^T Omega (k_i x p)
    const int gs0 = (int)P.groups.size();
    for (LT& lt : lts) {
      for (const LItem& li : lt.items) {
        if (li.dense) continue;
        begin_group(bscr(), li.sp_off, li.cap, li.k, dconst(lt.p), -1);
        add_item(li.zbuf, li.zoff, li.zld, FL_T, -1, 0, 0, FL_OMEGA, dconst(li.zrows), li.k, 0, 0,
                 (int)(1000003u * (uint32_t)(lt.node + 1)), li.col_off);
      }
    }
    stage(ST_GEMM, gs0, (int)P.groups.size(), TAG_S);

    // Y = sum_i coef_i X_i S_i   (dense items: X_i Omega[col rows])
    int g0 = (int)P.groups.size();
    for (LT& lt : lts) {
      const int m = S.cl[S.bn[lt.node].t].size;
      const int seed = (int)(1000003u * (uint32_t)(lt.node + 1));
      for (int r0 = 0; r0 < m; r0 += TILE) {
        int tr = std::min(TILE, m - r0);
        begin_group(bscr(), lt.y + r0, m, dconst(tr), dconst(lt.p), -1);
        for (const LItem& li : lt.items) {
          int a0 = std::max(li.row_off, r0), a1 = std::min(li.row_off + li.xrows, r0 + tr);
          if (a1 <= a0) continue;
          if (li.dense)
            add_item(li.xbuf, li.xoff + (a0 - li.row_off), li.xld, 0, -1, 0, 0, FL_OMEGA,
                     dconst(lsz), dconst(a1 - a0), a0 - r0, li.coef, seed, li.col_off, li.g0, li.g1);
          else
            add_item(li.xbuf, li.xoff + (a0 - li.row_off), li.xld, 0, bscr(), li.sp_off, li.cap, 0,
                     li.k, dconst(a1 - a0), a0 - r0, li.coef);
        }
      }
    }
    stage(ST_GEMM, g0, (int)P.groups.size(), TAG_Y);

    // orthonormal basis of range(Y): G = Y^T Y, pivoted Cholesky, Q = Y T
    auto orth_pass = [&](bool from_y) {
      int gg = (int)P.groups.size();
      for (size_t i = 0; i < lts.size(); ++i) {
        LT& lt = lts[i];
        const TInfo& ti = P.targets[i];
        int64_t src = from_y ? lt.y : lt.q;
        Dim pc = from_y ? dconst(lt.p) : drank(rscr(), ti.r_ri);
        begin_group(bscr(), ti.g_off, lt.p, pc, pc, -1);
        add_item(bscr(), src, ti.m, FL_T, bscr(), src, ti.m, 0, dconst(ti.m), pc, 0, 0);
      }
      stage(ST_GEMM, gg, (int)P.groups.size(), from_y ? TAG_G : TAG_G2);
      P.stages.push_back(Stage{ST_PCHOL, 0, (int)lts.size()});
      // record whether this pass truncates (first) or only re-orthogonalises
      if (!from_y) P.stages.back().kind = ST_PCHOL + 16;
      gg = (int)P.groups.size();
      for (size_t i = 0; i < lts.size(); ++i) {
        LT& lt = lts[i];
        const TInfo& ti = P.targets[i];
        int64_t src = from_y ? lt.y : lt.q;
        int64_t dst = from_y ? lt.q : lt.y;
        Dim pin = from_y ? dconst(lt.p) : drank(rscr(), ti.r_ri);
        for (int r0 = 0; r0 < ti.m; r0 += TILE) {
          int tr = std::min(TILE, ti.m - r0);
          begin_group(bscr(), dst + r0, ti.m, dconst(tr), drank(rscr(), ti.r_ri), -1);
          add_item(bscr(), src + r0, ti.m, 0, bscr(), ti.t_off, lt.p, 0, pin, dconst(tr), 0, 0);
        }
      }
      stage(ST_GEMM, gg, (int)P.groups.size(), from_y ? TAG_Q : TAG_Q2);
    };
    orth_pass(true);
    if (pp.cholqr2) {
      orth_pass(false);
      for (LT& lt : lts) std::swap(lt.y, lt.q);   // the basis now lives in the former Y buffer
    }

    // P_i = X_i^T Q[rows of i]   (k_i x r)
    g0 = (int)P.groups.size();
    for (size_t i = 0; i < lts.size(); ++i) {
      LT& lt = lts[i];
      const TInfo& ti = P.targets[i];
      for (const LItem& li : lt.items) {
        Dim kd = li.dense ? dconst(lsz) : li.k;
        begin_group(bscr(), li.sp_off, li.cap, kd, drank(rscr(), ti.r_ri), -1);
        add_item(li.xbuf, li.xoff, li.xld, FL_T, bscr(), lt.q + li.row_off, ti.m, 0,
                 dconst(li.xrows), kd, 0, 0);
      }
    }
    stage(ST_GEMM, g0, (int)P.groups.size(), TAG_P);

    // B^T = sum_i coef_i Z_i P_i   (n x r)
    g0 = (int)P.groups.size();
    for (size_t i = 0; i < lts.size(); ++i) {
      LT& lt = lts[i];
      const TInfo& ti = P.targets[i];
      for (int r0 = 0; r0 < ti.n; r0 += TILE) {
        int tr = std::min(TILE, ti.n - r0);
        begin_group(bscr(), lt.bt + r0, ti.n, dconst(tr), drank(rscr(), ti.r_ri), -1);
        for (const LItem& li : lt.items) {
          int a0 = std::max(li.col_off, r0), a1 = std::min(li.col_off + li.zrows, r0 + tr);
          if (a1 <= a0) continue;
          if (li.dense)
            add_item(-1, 0, 0, FL_IDENT, bscr(), li.sp_off + (a0 - li.col_off), li.cap, 0,
                     dconst(a1 - a0), dconst(a1 - a0), a0 - r0, li.coef, 0, 0, li.g0, li.g1);
          else
            add_item(li.zbuf, li.zoff + (a0 - li.col_off), li.zld, 0, bscr(), li.sp_off, li.cap, 0,
                     li.k, dconst(a1 - a0), a0 - r0, li.coef);
        }
      }
    }
    stage(ST_GEMM, g0, (int)P.groups.size(), TAG_BT);

    // H = (B^T)^T B^T   (r x r), core eigen-decomposition
    g0 = (int)P.groups.size();
    for (size_t i = 0; i < lts.size(); ++i) {
      const TInfo& ti = P.targets[i];
      Dim rr = drank(rscr(), ti.r_ri);
      begin_group(bscr(), ti.h_off, lts[i].p, rr, rr, -1);
      add_item(bscr(), lts[i].bt, ti.n, FL_T, bscr(), lts[i].bt, ti.n, 0, dconst(ti.n), rr, 0, 0);
    }
    stage(ST_GEMM, g0, (int)P.groups.size(), TAG_H);
    P.stages.push_back(Stage{ST_EIG, 0, (int)lts.size()});

    // U = Q W_k, V = B^T W_k into C
    g0 = (int)P.groups.size();
    for (size_t i = 0; i < lts.size(); ++i) {
      const TInfo& ti = P.targets[i];
      int lc = ti.c_leaf;
      Dim rr = drank(rscr(), ti.r_ri);
      for (int r0 = 0; r0 < ti.m; r0 += TILE) {
        int tr = std::min(TILE, ti.m - r0);
        begin_group(bU(cr), S.lr_row0[lc] * kc + r0, ti.m, dconst(tr), drank(cr, lc), -1);
        add_item(bscr(), lts[i].q + r0, ti.m, 0, bscr(), ti.w_off, lts[i].p, 0, rr, dconst(tr), 0, 0);
      }
      for (int r0 = 0; r0 < ti.n; r0 += TILE) {
        int tr = std::min(TILE, ti.n - r0);
        begin_group(bV(cr), S.lr_col0[lc] * kc + r0, ti.n, dconst(tr), drank(cr, lc), -1);
        add_item(bscr(), lts[i].bt + r0, ti.n, 0, bscr(), ti.w_off, lts[i].p, 0, rr, dconst(tr), 0, 0);
      }
    }
    stage(ST_GEMM, g0, (int)P.groups.size(), TAG_UV);
    (void)capsum_max;
  }
};

}  // namespace

namespace {
// Order every GEMM stage's groups wide (static 64-column outputs) first and
// record their count, so a launch can give the two kinds different kernels.
// Groups of one stage write disjoint outputs: their order changes nothing.
// Also records the widest sketch of the plan's targets.
void order_wide_first(Plan& plan) {
  plan.max_p = 0;
  for (const TInfo& ti : plan.targets) plan.max_p = std::max(plan.max_p, ti.p);
  for (Stage& sg : plan.stages) {
    if (sg.kind != ST_GEMM) continue;
    auto wide = [](const GGroup& g) { return g.n_rb < 0 && g.n_st >= 64; };
    auto mid = std::stable_partition(plan.groups.begin() + sg.beg, plan.groups.begin() + sg.end,
                                     wide);
    sg.nwide = (int)(mid - (plan.groups.begin() + sg.beg));
  }
}
}  // namespace

void build_plan(const Structure& S, const OpDesc& op, const PlanParams& pp, Plan& plan) {
  plan = Plan();
  plan.nroles = op.nroles;
  Builder b(S, op, pp, plan);
  const BNode& c = S.bn[op.c_node];
  for (int pi = 0; pi < (int)op.prods.size(); ++pi) {
    const OpDesc::Prod& pr = op.prods[pi];
    const BNode& a = S.bn[pr.a_node];
    const BNode& bb = S.bn[pr.b_node];
    if (a.t != c.t || bb.s != c.s || a.s != bb.t)
      throw std::runtime_error("product operands do not conform with the target block");
    b.mm(pi, a.t, a.s, bb.s);
  }
  plan.n_terms = (int)b.terms.size();
  b.phase1();
  b.phase2();
  order_wide_first(plan);
}

namespace {
// canonical position of a stage in every plan
int stage_slot(const Stage& sg) {
  if (sg.kind == ST_GEMM) {
    static const int slot_of_tag[NTAGS] = {0, 1, 2, 3, 4, 5, 7, 8, 10, 11, 12, 13, 15};
    return slot_of_tag[sg.tag];
  }
  if (sg.kind == ST_PCHOL) return 6;
  if (sg.kind == ST_PCHOL + 16) return 9;
  return 14;   // ST_EIG
}
}  // namespace

void merge_plans(const std::vector<const Plan*>& ps, Plan& out) {
  out = Plan();
  const int nr = ps[0]->nroles;
  out.nroles = nr;
  const int sb = 3 * nr, rb = nr;
  std::vector<int64_t> soff(ps.size());
  std::vector<int> roff(ps.size()), toff(ps.size());
  for (size_t i = 0; i < ps.size(); ++i) {
    soff[i] = out.scratch;
    roff[i] = out.scratch_ranks;
    toff[i] = (int)out.targets.size();
    out.scratch += ps[i]->scratch;
    out.scratch_ranks += ps[i]->scratch_ranks;
    const int sk0 = (int)out.stack.size();
    out.stack.insert(out.stack.end(), ps[i]->stack.begin(), ps[i]->stack.end());
    for (TInfo ti : ps[i]->targets) {
      ti.g_off += soff[i]; ti.t_off += soff[i]; ti.h_off += soff[i]; ti.w_off += soff[i];
      ti.r_ri += roff[i];
      ti.sk_beg += sk0; ti.sk_end += sk0;
      out.targets.push_back(ti);
    }
    out.n_lr_targets += ps[i]->n_lr_targets;
    out.n_dense_targets += ps[i]->n_dense_targets;
    out.n_terms += ps[i]->n_terms;
    out.flops_static += ps[i]->flops_static;
  }
  for (int slot = 0; slot < 16; ++slot) {
    int kind = -1, tag = -1, g0 = (int)out.groups.size(), tb = -1, te = -1;
    for (size_t i = 0; i < ps.size(); ++i) {
      for (const Stage& sg : ps[i]->stages) {
        if (stage_slot(sg) != slot) continue;
        kind = sg.kind;
        tag = sg.tag;
        if (sg.kind == ST_GEMM) {
          for (int g = sg.beg; g < sg.end; ++g) {
            GGroup G = ps[i]->groups[g];
            const int ib = (int)out.items.size();
            for (int it = G.ib; it < G.ie; ++it) {
              GItem I = ps[i]->items[it];
              if (I.abuf == sb) I.aoff += soff[i];
              if (I.bbuf == sb) I.boff += soff[i];
              if (I.k_rb == rb) I.k_ri += roff[i];
              if (I.r_rb == rb) I.r_ri += roff[i];
              out.items.push_back(I);
            }
            G.ib = ib;
            G.ie = (int)out.items.size();
            if (G.cbuf == sb) G.coff += soff[i];
            if (G.m_rb == rb) G.m_ri += roff[i];
            if (G.n_rb == rb) G.n_ri += roff[i];
            out.groups.push_back(G);
          }
        } else {
          const int b = sg.beg + toff[i], e = sg.end + toff[i];
          tb = tb < 0 ? b : std::min(tb, b);
          te = std::max(te, e);
        }
      }
    }
    if (kind < 0) continue;
    if (kind == ST_GEMM) {
      if ((int)out.groups.size() > g0) out.stages.push_back(Stage{kind, g0, (int)out.groups.size(), tag});
    } else if (te > tb) {
      out.stages.push_back(Stage{kind, tb, te, -1});
    }
  }
  order_wide_first(out);
}

void MatvecPlan::build(const Structure& S) {
  const int nc = S.nleafcl, lsz = S.lsz;
  std::vector<std::vector<int>> dr(nc), dc(nc), lr(nc), lc(nc);
  std::vector<std::vector<int>> dro(nc), dco(nc), lro(nc), lco(nc);
  lr_m.assign(S.lleaf.size(), 0); lr_n = lr_m; lr_t0 = lr_m; lr_s0 = lr_m;
  for (size_t i = 0; i < S.lleaf.size(); ++i) {
    const BNode& b = S.bn[S.lleaf[i]];
    const Cluster &ct = S.cl[b.t], &cs = S.cl[b.s];
    lr_m[i] = ct.size; lr_n[i] = cs.size; lr_t0[i] = ct.begin; lr_s0[i] = cs.begin;
    for (int r = ct.begin; r < ct.begin + ct.size; r += lsz) {
      lr[r / lsz].push_back((int)i);
      lro[r / lsz].push_back(r - ct.begin);
    }
    for (int q = cs.begin; q < cs.begin + cs.size; q += lsz) {
      lc[q / lsz].push_back((int)i);
      lco[q / lsz].push_back(q - cs.begin);
    }
  }
  for (size_t d = 0; d < S.dleaf.size(); ++d) {
    const BNode& b = S.bn[S.dleaf[d]];
    const Cluster &ct = S.cl[b.t], &cs = S.cl[b.s];
    dr[ct.begin / lsz].push_back((int)d);
    dro[ct.begin / lsz].push_back(cs.begin);
    dc[cs.begin / lsz].push_back((int)d);
    dco[cs.begin / lsz].push_back(ct.begin);
  }
  auto csr = [&](std::vector<std::vector<int>>& a, std::vector<std::vector<int>>& b,
                 std::vector<int32_t>& ptr, std::vector<int32_t>& x, std::vector<int32_t>& y) {
    ptr.assign(nc + 1, 0);
    x.clear(); y.clear();
    for (int c = 0; c < nc; ++c) {
      ptr[c + 1] = ptr[c] + (int)a[c].size();
      x.insert(x.end(), a[c].begin(), a[c].end());
      y.insert(y.end(), b[c].begin(), b[c].end());
    }
  };
  csr(dr, dro, d_ptr, d_leaf, d_col);
  csr(lr, lro, l_ptr, l_leaf, l_rowoff);
  csr(dc, dco, dt_ptr, dt_leaf, dt_row);
  csr(lc, lco, lt_ptr, lt_leaf, lt_coloff);
  auto segs = [&](const std::vector<int32_t>& rows, std::vector<int32_t>& ptr) {
    ptr.assign(rows.size() + 1, 0);
    for (size_t l = 0; l < rows.size(); ++l) ptr[l + 1] = ptr[l] + (rows[l] + lsz - 1) / lsz;
  };
  segs(lr_n, seg_ptr);
  segs(lr_m, segt_ptr);
}

}  // namespace acr
