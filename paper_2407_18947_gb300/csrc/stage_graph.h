// Recording of one RT-CC3 residual evaluation on the engine tape.
//
// Conventions (closed shell, occupied orbitals first, n = o + v):
//   g[p,q,r,s] = (pq|rs)~  dressed chemists' integrals; the paper's <pq|rs> is (pr|qs)
//   t1[i,a] = t_i^a, t2[i,j,a,b] = t_ij^ab, t3[i,j,k,a,b,c] = t_ijk^abc  (Eqs. A17-A19)
//   w = beta V = -E(t) . mu (Eq. 1, Eq. 10)
// The T residuals are R1 = <mu1|H + [H,T2] + [H,T3]|0>, R2 = <mu2|... + 1/2[[H,T2],T2]|0>
// (Eqs. A10-A11) with H the T1-transformed Hamiltonian (Eq. 8, Eq. A4) and t3 the
// solution of the triples equation Eq. 4 / Eq. A12 with dt3/dt = 0.
#pragma once

#include "model.h"
#include "rotation.h"

namespace rtcc3 {

// Field-dressed eigenbasis of one stage (see rotation.h): O and V are built
// from the dressed perturbation and decomposed on the engine's side stream,
// overlapping the CCSD part of the stage; rotated_triples joins before use.
template <typename R>
struct FieldBasis {
  int So = -1, Sio = -1, Sv = -1, Siv = -1;  // S and S^-1 (compute precision)
  Cx<R>* osum = nullptr;                     // eigenvalue sums (compute precision)
  Cx<R>* vsum = nullptr;
};

// `ahead` (optional): the decomposition was enqueued on the side stream before
// this stage (see launch_next_field_matrices); only the conversions remain.
template <typename R>
FieldBasis<R> start_field_basis(Engine<R>& E, const Hamil<R>& H, int wt,
                                const BasisBuffers* ahead = nullptr) {
  const int o = H.o, v = H.v;
  Arena& A = E.arena();
  auto c2 = [&](size_t n) { return static_cast<double2*>(A.alloc(sizeof(double2) * n)); };
  // the arena layout does not depend on `ahead`
  BasisBuffers bb;
  bb.Mo = c2(size_t(o) * o);
  bb.Mv = c2(size_t(v) * v);
  bb.So = c2(size_t(o) * o);
  bb.Sio = c2(size_t(o) * o);
  bb.Sv = c2(size_t(v) * v);
  bb.Siv = c2(size_t(v) * v);
  bb.lo = c2(o);
  bb.lv = c2(v);
  bb.wso = c2(3 * size_t(o) * o);
  bb.wsv = c2(3 * size_t(v) * v);
  if (ahead) bb = *ahead;
  double2 *So64 = bb.So, *Sio64 = bb.Sio, *Sv64 = bb.Sv, *Siv64 = bb.Siv, *lo = bb.lo, *lv = bb.lv;
  FieldBasis<R> B;
  B.osum = static_cast<Cx<R>*>(A.alloc(sizeof(Cx<R>) * size_t(o) * o * o));
  B.vsum = static_cast<Cx<R>*>(A.alloc(sizeof(Cx<R>) * size_t(v) * v * v));
  B.So = E.node({o, o}, false, false);
  B.Sio = E.node({o, o}, false, false);
  B.Sv = E.node({v, v}, false, false);
  B.Siv = E.node({v, v}, false, false);
  int* status = E.error_flag();
  E.fork();
  const cudaStream_t ss = E.side_stream();
  const int pk = E.prof_begin(ss);
  if (!ahead) {
    launch_field_matrices<R>(E.data(wt), H.eps, o, v, bb.Mo, bb.Mv, ss);
    const EigJob jo{bb.Mo, o, So64, Sio64, lo, bb.wso, E.eig_sweep_cap()};
    const EigJob jv{bb.Mv, v, Sv64, Siv64, lv, bb.wsv, E.eig_sweep_cap()};
    launch_eig(jo, jv, sizeof(R) == 4, status, ss);
  }
  launch_lambda_sums<R>(lo, lv, o, v, H.eshift, B.osum, B.vsum, ss);
  launch_to_precision<R>(So64, E.data(B.So), size_t(o) * o, ss);
  launch_to_precision<R>(Sio64, E.data(B.Sio), size_t(o) * o, ss);
  launch_to_precision<R>(Sv64, E.data(B.Sv), size_t(v) * v, ss);
  launch_to_precision<R>(Siv64, E.data(B.Siv), size_t(v) * v, ss);
  E.prof_end(pk, ss, "field_eig", 0.0, 0.0);
  E.add_launches(ahead ? 5 : 7);
  return B;
}

// ---- Blocked triples: W and t3 recomputed per slab, never stored --------------
//
// The operands of the connected triples and of their contractions into X1 and
// X2 (already in the basis in which the denominators are diagonal):
//   Z[ijkabc] = sum_E Ac[i,j,a,E] Bc[E,k,b,c] - sum_m T2[i,m,a,b] G2[m,j,c,k]
//   t3 = -P_ijk^abc(Z) / D                                  (Eqs. A25, A30, 6)
//   X1[i,a]     = sum (t3 - t3(ijkcba)) Lp[j,k,b,c]              (Eq. A21)
//   S3[i,j,a,b] = sum (t3 - t3(ijkcba)) Fp[k,c]
//               + sum (2 t3 - t3(ijkacb) - t3(ijkcba))[ijk cbe] Gb[a,c,k,e]
//               - sum (2 t3 - t3(mjkbac) - t3(mjkcba))[mjk cba] Gc[k,i,m,c]
// (X2 = P_ij^ab S3, Eq. A22).  The (i,j,k) blocks are processed in slabs of
// `chunk` first occupied indices (the paper's per-(i,j,k) evaluation with the
// v^3 blocks of several (i,j,k) grouped into one slab, Section 2.1).
template <typename R>
struct TriplesOperands {
  View Ac, Bc, T2, G2, Lp, Fp, Gb, Gc;
};

// Field-coupling adjoint in the rotated basis: grad(v~_vv) -= S_v^-T D'_vv S_v^T,
// grad(v~_oo) += S_o D'_oo S_o^-1 with the slot densities D' of y' = grad(t3')/D'
// and t3' (the triples density terms of Eqs. A31-A32 in the rotated basis).
struct FieldAdjoint {
  bool on = false;
  int wt = -1;
  View wvv, woo, SO, SIO, SV, SIV;
};

// Forward: for each slab, W = P_ijk^abc Z from the three Z slabs with the
// slab's index i in each of the three occupied positions, t3 = -W / D,
// and its contributions to X1 (rows of the slab) and S3.  Reverse (custom
// adjoint, given grad X1 and grad S3): per slab, t3 is rebuilt; the
// cotangents of Lp, Fp, Gb, Gc follow from t3; the t3 cotangent Q is
// needed symmetrised, P_ijk^abc(Q) = R + R(ikjacb) with R the sum of Q
// evaluated with the slab index in each of the three occupied positions
// (Q is a sum of products of small tensors, so any arrangement is cheap to
// form); Z's cotangent is -P(Q)/D, which gives those of Ac, Bc, T2, G2, and
// with t3 the field-coupling slot densities.  Memory: four slabs of
// chunk * o^2 v^3 elements instead of the dozen o^3 v^3 tensors of the stored
// form.  X1o, S3o: output nodes (written here, zero-initialised).
template <typename R>
void blocked_triples(Engine<R>& E, int o, int v, int chunk, const TriplesOperands<R>& in,
                     const typename Engine<R>::EpsSpec& es, int X1o, int S3o,
                     const FieldAdjoint& fa) {
  const int I0 = std::max(1, std::min(chunk, o));
  const bool g = E.needs_grad(in.Ac.node) || E.needs_grad(in.Bc.node) ||
                 E.needs_grad(in.T2.node) || E.needs_grad(in.G2.node) ||
                 E.needs_grad(in.Lp.node) || E.needs_grad(in.Fp.node) ||
                 E.needs_grad(in.Gb.node) || E.needs_grad(in.Gc.node) ||
                 (fa.on && E.needs_grad(fa.wt));
  // slab buffers: nb0 holds t3; nb1..nb3 hold the three Z slabs while W is
  // built, then serve as scratch (nb1) and P(Q)/D (nb2) in the reverse pass
  const int nb0 = E.node({I0, o, o, v, v, v}, false, false);
  const int nb1 = E.node({I0, o, o, v, v, v}, false, false);
  const int nb2 = E.node({I0, o, o, v, v, v}, false, false);
  const int nb3 = E.node({I0, o, o, v, v, v}, false, false);
  E.set_needs_grad(X1o, g);
  E.set_needs_grad(S3o, g);

  // slab view (I rows) of a slab node
  auto slab = [&E](int nb, int I) { return E.v(nb).sub(0, 0, I); };
  // One product of the slab loop.  The letter i is the slab's index: a slab
  // view (s = true) holds the slab's rows already; any other operand that
  // carries i is sliced to the slab (view at start 0 plus the start as a
  // pointer shift, so that all slabs of one extent share one plan).
  struct Arg { View v; bool g; bool s; };
  auto prod = [&E](const std::string& spec, double alpha, Arg a, Arg b, Arg c, int i0, int I,
                   bool acc) {
    const size_t comma = spec.find(','), arrow = spec.find("->");
    const std::string sa = spec.substr(0, comma), sb = spec.substr(comma + 1, arrow - comma - 1),
                      sc = spec.substr(arrow + 2);
    long long sh[3] = {0, 0, 0};
    Arg* ops[3] = {&a, &b, &c};
    const std::string* lets[3] = {&sa, &sb, &sc};
    for (int w = 0; w < 3; ++w) {
      const size_t d = lets[w]->find('i');
      if (d == std::string::npos || ops[w]->s) continue;
      sh[w] = (long long)i0 * ops[w]->v.stride[d];
      ops[w]->v = ops[w]->v.sub(int(d), 0, I);
    }
    E.exec_contract_at(spec.c_str(), alpha, a.v, a.g, sh[0], b.v, b.g, sh[1], c.v, c.g, sh[2], acc);
  };
  // t3 of the slab into T.  The three Z slabs with the slab index in each
  // occupied position, Z1[i,j,k,..] = Z[i,j,k,..], Z2[i,j,k,..] = Z[j,i,k,..]
  // and Z3[i,j,k,..] = Z[j,k,i,..] (two products each), then
  // W = Z1 + Z1(ikjacb) + Z2(ijkbac) + Z2(ikjcab) + Z3(ikjcba) + Z3(ijkbca)
  // (the six terms of P_ijk^abc) in one pass, and t3 = -W / D.
  auto build_t3 = [&E, prod, in, es](const View& T, const View& Z1, const View& Z2, const View& Z3,
                                     int i0, int I) {
    const View* Zs[3] = {&Z1, &Z2, &Z3};
    static const char* kA[3] = {"ijaE,Ekbc->ijkabc", "jiaE,Ekbc->ijkabc", "jkaE,Eibc->ijkabc"};
    static const char* kB[3] = {"imab,mjck->ijkabc", "jmab,mick->ijkabc", "jmab,mkci->ijkabc"};
    for (int p = 0; p < 3; ++p) {
      prod(kA[p], 1.0, {in.Ac, false, false}, {in.Bc, false, false}, {*Zs[p], false, true}, i0, I,
           false);
      prod(kB[p], -1.0, {in.T2, false, false}, {in.G2, false, false}, {*Zs[p], false, true}, i0, I,
           true);
    }
    E.exec_combine({{1.0, Z1}, {1.0, E.ev("ikjacb->ijkabc", Z1)}, {1.0, E.ev("ijkbac->ijkabc", Z2)},
                    {1.0, E.ev("ikjcab->ijkabc", Z2)}, {1.0, E.ev("ikjcba->ijkabc", Z3)},
                    {1.0, E.ev("ijkbca->ijkabc", Z3)}},
                   T, true);
    E.exec_slab_div(-1.0, T, i0, es, T);
  };
  const View X1v = E.v(X1o), S3v = E.v(S3o);
  for (int i0 = 0; i0 < o; i0 += I0) {
    const int I = std::min(I0, o - i0);
    const View T = slab(nb0, I), U = slab(nb1, I);
    build_t3(T, U, slab(nb2, I), slab(nb3, I), i0, I);
    E.exec_combine({{1.0, T}, {-1.0, E.ev("ijkcba->ijkabc", T)}}, U, true);
    prod("ijkabc,jkbc->ia", 1.0, {U, false, true}, {in.Lp, false, false}, {X1v, false, false}, i0, I, true);
    prod("ijkabc,kc->ijab", 1.0, {U, false, true}, {in.Fp, false, false}, {S3v, false, false}, i0, I, true);
    E.exec_combine({{2.0, T}, {-1.0, E.ev("ijkxzy->ijkxyz", T)}, {-1.0, E.ev("ijkzyx->ijkxyz", T)}},
                   U, true);
    prod("ijkcbe,acke->ijab", 1.0, {U, false, true}, {in.Gb, false, false}, {S3v, false, false}, i0, I, true);
    E.exec_combine({{2.0, T}, {-1.0, E.ev("ijkyxz->ijkxyz", T)}, {-1.0, E.ev("ijkzyx->ijkxyz", T)}},
                   U, true);
    // the slab index is Uc's first occupied index (m), a sum index here
    prod("imkcba,kjic->jmab", -1.0, {U, false, true}, {in.Gc, false, false}, {S3v, false, false}, i0, I, true);
  }
  if (!g) return;
  const int Gb2 = E.node({v, v, o, v}, false, false);
  E.exec_combine({{2.0, in.Gb}, {-1.0, E.ev("dzrx->dxrz", in.Gb)}}, E.v(Gb2), true);
  const View GB2 = E.v(Gb2);
  E.custom([&E, o, v, I0, in, es, fa, nb0, nb1, nb2, nb3, X1o, S3o, GB2, prod, build_t3, slab]() {
    const View X1v = E.v(X1o), S3v = E.v(S3o);
    const bool gl = E.needs_grad(in.Lp.node), gf = E.needs_grad(in.Fp.node),
               gb = E.needs_grad(in.Gb.node), gc = E.needs_grad(in.Gc.node);
    const bool gfield = fa.on && E.needs_grad(fa.wt);
    int Dv = -1, Do = -1;
    if (gfield) {
      Dv = E.node({v, v});
      Do = E.node({o, o});
    }
    // Q[p,q,r,x,y,z] (the t3 cotangent) as nine products of small tensors;
    // placeholders p q r x y z are mapped to the output letters of one of
    // the three arrangements, d and l are sums
    struct QT { const char* a; int ga; const char* b; double alpha; };
    // ga: 0 grad X1, 1 grad S3; b operand: 0 Lp, 1 Fp, 2 Gb2, 3 Gb, 4 Gc
    static const char* kQa[9] = {"px", "pqxy", "pz", "pqzy", "pqdy", "pqdz", "lqzy", "lqzx", "lqxy"};
    static const int kQga[9] = {0, 1, 0, 1, 1, 1, 1, 1, 1};
    static const char* kQb[9] = {"qryz", "rz", "qryx", "rx", "dxrz", "dxry", "rlpx", "rlpy", "rlpz"};
    static const int kQbw[9] = {0, 1, 0, 1, 2, 3, 4, 4, 4};
    static const double kQal[9] = {1.0, 1.0, -1.0, -1.0, 1.0, -1.0, -2.0, 1.0, 1.0};
    static const char* kPos[3] = {"ijkabc", "jikbac", "kjicba"};  // p q r x y z
    const View bops[5] = {in.Lp, in.Fp, GB2, in.Gb, in.Gc};
    auto map = [](const char* t, const char* pos) {
      std::string r(t);
      for (char& ch : r) {
        const char* ph = "pqrxyz";
        for (int k = 0; k < 6; ++k)
          if (ch == ph[k]) { ch = pos[k]; break; }
      }
      return r;
    };
    for (int i0 = 0; i0 < o; i0 += I0) {
      const int I = std::min(I0, o - i0);
      const View T = slab(nb0, I), U = slab(nb1, I), W = slab(nb2, I);
      build_t3(T, U, W, slab(nb3, I), i0, I);
      // cotangents of the X-side operands
      if (gl || gf) {
        E.exec_combine({{1.0, T}, {-1.0, E.ev("ijkcba->ijkabc", T)}}, U, true);
        if (gl) prod("ijkabc,ia->jkbc", 1.0, {U, false, true}, {X1v, true, false}, {in.Lp, true, false}, i0, I, true);
        if (gf) prod("ijkabc,ijab->kc", 1.0, {U, false, true}, {S3v, true, false}, {in.Fp, true, false}, i0, I, true);
      }
      if (gb) {
        E.exec_combine({{2.0, T}, {-1.0, E.ev("ijkxzy->ijkxyz", T)},
                        {-1.0, E.ev("ijkzyx->ijkxyz", T)}}, U, true);
        prod("ijkcbe,ijab->acke", 1.0, {U, false, true}, {S3v, true, false}, {in.Gb, true, false}, i0, I, true);
      }
      if (gc) {
        E.exec_combine({{2.0, T}, {-1.0, E.ev("ijkyxz->ijkxyz", T)},
                        {-1.0, E.ev("ijkzyx->ijkxyz", T)}}, U, true);
        prod("imkcba,jmab->kjic", -1.0, {U, false, true}, {S3v, true, false}, {in.Gc, true, false}, i0, I, true);
      }
      // R = sum over the three arrangements of Q; S = R + R(ikjacb) = P(Q)
      bool first = true;
      for (int ps = 0; ps < 3; ++ps)
        for (int t = 0; t < 9; ++t) {
          const std::string spec = map(kQa[t], kPos[ps]) + "," + map(kQb[t], kPos[ps]) + "->ijkabc";
          prod(spec, kQal[t], {kQga[t] ? S3v : X1v, true, false}, {bops[kQbw[t]], false, false}, {U, false, true}, i0,
               I, !first);
          first = false;
        }
      E.exec_combine({{1.0, U}, {1.0, E.ev("ikjacb->ijkabc", U)}}, W, true);
      E.exec_slab_div(1.0, W, i0, es, W);  // W = P(Q) / D = -grad Z
      if (gfield) {
        // slot densities of the symmetrised y' = P(Q) / (6 D) with t3,
        // summed over the three slots: 1/2 of one slot of P(Q) / D
        E.branch_begin();
        E.exec_contract_at("jkiabc,jklabc->li", 0.5, W, false, 0, T, false, 0, E.v(Do), false, 0,
                           true);
        E.branch_switch();
        E.exec_contract_at("ijkabc,ijkdbc->ad", 0.5, W, false, 0, T, false, 0, E.v(Dv), false, 0,
                           true);
        E.branch_join();
      }
      if (E.needs_grad(in.Ac.node))
        prod("ijkabc,Ekbc->ijaE", -1.0, {W, false, true}, {in.Bc, false, false}, {in.Ac, true, false}, i0, I, true);
      if (E.needs_grad(in.Bc.node))
        prod("ijaE,ijkabc->Ekbc", -1.0, {in.Ac, false, false}, {W, false, true}, {in.Bc, true, false}, i0, I, true);
      if (E.needs_grad(in.T2.node))
        prod("ijkabc,mjck->imab", 1.0, {W, false, true}, {in.G2, false, false}, {in.T2, true, false}, i0, I, true);
      if (E.needs_grad(in.G2.node))
        prod("imab,ijkabc->mjck", 1.0, {in.T2, false, false}, {W, false, true}, {in.G2, true, false}, i0, I, true);
    }
    if (gfield) {
      const int tv = E.node({v, v}), to = E.node({o, o});
      E.exec_contract("Aa,AD->aD", 1.0, fa.SIV, false, E.v(Dv), false, E.v(tv), false);
      E.exec_contract("aD,dD->ad", -1.0, E.v(tv), false, fa.SV, false, fa.wvv, true);
      E.exec_contract("lL,LI->lI", 1.0, fa.SO, false, E.v(Do), false, E.v(to), false);
      E.exec_contract("lI,Ii->li", 1.0, E.v(to), false, fa.SIO, false, fa.woo, true);
    }
  }, true);
}

// Triples with the field coupling in the field-dressed eigenbasis (see
// rotation.h).  Forward: with the eigenbasis of O and V of this stage (from
// start_field_basis), rotate the inputs of W and of the source
// 1/2[[V~,T2],T2], divide by the complex denominators, form X1 and X2 in the
// rotated basis and rotate them back.  The rotations are constants of the
// tape (A^-1 does not depend on the choice of eigenbasis); the dependence of
// A on v~ is added by a custom adjoint: with y' = grad(t3') / D',
// grad(v~_vv) -= S_v^-T D'_vv S_v^T and grad(v~_oo) += S_o D'_oo S_o^-1, the
// slot densities D' of y' and t3' (the triples density terms of Eqs. A31-A32
// in the rotated basis).  Returns the node of t3' and accumulates into R1 and SD.
template <typename R, typename BlkFn>
int rotated_triples(Engine<R>& E, const Hamil<R>& H, const View& T, int wt, const FieldBasis<R>& B,
                    int g, int ft, const View& R1, const View& SD, BlkFn&& blk, int chunk = 0) {
  const int o = H.o, v = H.v;
  E.join();
  const int So = B.So, Sio = B.Sio, Sv = B.Sv, Siv = B.Siv;
  const View SO = E.v(So), SIO = E.v(Sio), SV = E.v(Sv), SIV = E.v(Siv);
  auto G = [&](const char* b) { return blk(g, b); };
  // rotate one index of a 4-index tensor: spec like "Ii,ijae->Ijae"
  auto rot = [&](const char* spec, const View& S, const View& X, const std::vector<int>& shape) {
    const int out = E.node(shape, false, false);  // first write overwrites: no zero fill
    E.contract(spec, 1.0, S, X, E.v(out), false);
    return E.v(out);
  };
  const std::vector<int> s6 = {o, o, o, v, v, v};
  // ---- rotated inputs of W: indices that become indices of t3 take S^-1 --------
  View T1p = rot("Ii,ijae->Ijae", SIO, T, {o, o, v, v});
  T1p = rot("Jj,Ijae->IJae", SIO, T1p, {o, o, v, v});
  T1p = rot("Aa,IJae->IJAe", SIV, T1p, {o, o, v, v});
  View G1p = rot("Cc,ckbe->Ckbe", SIV, G("vovv"), {v, o, v, v});
  G1p = rot("Kk,Ckbe->CKbe", SIO, G1p, {v, o, v, v});
  G1p = rot("Bb,CKbe->CKBe", SIV, G1p, {v, o, v, v});
  View T2p = rot("Ii,imab->Imab", SIO, T, {o, o, v, v});
  T2p = rot("Aa,Imab->ImAb", SIV, T2p, {o, o, v, v});
  T2p = rot("Bb,ImAb->ImAB", SIV, T2p, {o, o, v, v});
  View G2p = rot("Jj,mjck->mJck", SIO, G("oovo"), {o, o, v, o});
  G2p = rot("Cc,mJck->mJCk", SIV, G2p, {o, o, v, o});
  G2p = rot("Kk,mJCk->mJCK", SIO, G2p, {o, o, v, o});
  // source -P sum_ld v~_ld t_ij^ad t_kl^cb, rotated the same way; P is linear,
  // so it is folded into Z before the one permutation sum
  const int Yl = E.node({o, o, o, v}, false, false);
  E.contract("ld,ijad->lija", 1.0, blk(wt, "ov"), T, E.v(Yl), false);
  View Ylp = rot("Ii,lija->lIja", SIO, E.v(Yl), {o, o, o, v});
  Ylp = rot("Jj,lIja->lIJa", SIO, Ylp, {o, o, o, v});
  Ylp = rot("Aa,lIJa->lIJA", SIV, Ylp, {o, o, o, v});
  View T3p_ = rot("Kk,klcb->Klcb", SIO, T, {o, o, v, v});
  T3p_ = rot("Cc,Klcb->KlCb", SIV, T3p_, {o, o, v, v});
  T3p_ = rot("Bb,KlCb->KlCB", SIV, T3p_, {o, o, v, v});
  // Z = sum_e t'_ij^ae g'_ckbe - sum_m t'_im^ab g'_mjck - sum_l y'_lija t'_kl^cb:
  // the first and last terms group Z's indices the same way ((ija) x (kbc)),
  // so they are one product over the concatenated sum index E = (e | l)
  // (one pass over Z instead of two, and one reverse product per operand)
  const int Ac = E.node({o, o, v, v + o}, false, false);
  E.combine({{1.0, T1p}}, E.v(Ac).sub(3, 0, v), true);
  E.combine({{-1.0, E.ev("lija->ijal", Ylp)}}, E.v(Ac).sub(3, v, o), true);
  const int Bc = E.node({v + o, o, v, v}, false, false);
  E.combine({{1.0, E.ev("ckbe->ekbc", G1p)}}, E.v(Bc).sub(0, 0, v), true);
  E.combine({{1.0, E.ev("klcb->lkbc", T3p_)}}, E.v(Bc).sub(0, v, o), true);
  // ---- X-side operands in the rotated basis: contracted indices take S
  // (contravariant), free rotated indices S^-1 ------------------------------------
  const int Ljk = E.node({o, o, v, v}, false, false);
  E.combine({{2.0, E.ev("jbkc->jkbc", G("ovov"))}, {-1.0, E.ev("jckb->jkbc", G("ovov"))}},
            E.v(Ljk), true);
  View Lp = rot("jJ,jkbc->Jkbc", SO, E.v(Ljk), {o, o, v, v});
  Lp = rot("kK,Jkbc->JKbc", SO, Lp, {o, o, v, v});
  Lp = rot("bB,JKbc->JKBc", SV, Lp, {o, o, v, v});
  Lp = rot("cC,JKBc->JKBC", SV, Lp, {o, o, v, v});
  View Fp = rot("kK,kc->Kc", SO, blk(ft, "ov"), {o, v});
  Fp = rot("cC,Kc->KC", SV, Fp, {o, v});
  View Gb = rot("Aa,acke->Acke", SIV, G("vvov"), {v, v, o, v});
  Gb = rot("cC,Acke->ACke", SV, Gb, {v, v, o, v});
  Gb = rot("kK,ACke->ACKe", SO, Gb, {v, v, o, v});
  Gb = rot("eE,ACKe->ACKE", SV, Gb, {v, v, o, v});
  View Gc = rot("kK,kimc->Kimc", SO, G("ooov"), {o, o, o, v});
  Gc = rot("Ii,Kimc->KImc", SIO, Gc, {o, o, o, v});
  Gc = rot("mM,KImc->KIMc", SO, Gc, {o, o, o, v});
  Gc = rot("cC,KIMc->KIMC", SV, Gc, {o, o, o, v});
  typename Engine<R>::EpsSpec es;
  es.o = o;
  es.v = v;
  es.osum_cr = B.osum;
  es.vsum_cr = B.vsum;
  es.order = H.orbit_order;
  const int X1p = E.node({o, v}, false, chunk > 0);
  const int S3p = E.node({o, o, v, v}, false, chunk > 0);
  int t3p = -1;
  if (chunk > 0) {
    // blocked: W and t3' per slab of occupied indices, never stored
    FieldAdjoint fa;
    fa.on = true;
    fa.wt = wt;
    fa.wvv = blk(wt, "vv");
    fa.woo = blk(wt, "oo");
    fa.SO = SO;
    fa.SIO = SIO;
    fa.SV = SV;
    fa.SIV = SIV;
    blocked_triples<R>(E, o, v, chunk, {E.v(Ac), E.v(Bc), T2p, G2p, Lp, Fp, Gb, Gc}, es, X1p,
                       S3p, fa);
  } else {
  const int Z = E.node(s6, false, false);
  E.contract("ijaE,Ekbc->ijkabc", 1.0, E.v(Ac), E.v(Bc), E.v(Z), false);
  E.contract("imab,mjck->ijkabc", -1.0, T2p, G2p, E.v(Z), true);
  // ---- t3' = -P(Z) / D' with the complex denominators ---------------------------
  t3p = E.node(s6, false, false);
  const int wtn = wt;
  // with the field adjoint below, it also takes over the reverse of the
  // symmetrised division: both read the six permutations of grad(t3'), so
  // grad(Z) and ys come from one pass
  const bool pair = E.needs_grad(Z) && E.needs_grad(wtn);
  if (pair) {
    E.exec_sym6_div(-1.0, E.v(Z), es, E.v(t3p));
    E.set_needs_grad(t3p, true);
  } else {
    E.sym6_div(-1.0, E.v(Z), es, E.v(t3p));
  }
  if (E.needs_grad(t3p) && E.needs_grad(wtn)) {
    const View wvv = blk(wt, "vv"), woo = blk(wt, "oo");
    E.custom([&E, t3p, wtn, Z, pair, es, s6, SO, SIO, SV, SIV, wvv, woo, o, v]() {
      if (!E.needs_grad(t3p) || !E.needs_grad(wtn)) return;
      const View T3 = E.v(t3p);
      // y' = grad(t3') / D'; t3' is invariant under the simultaneous
      // permutations, so the slot-2 and slot-3 densities of y' equal the
      // slot-1 densities of the permuted y': ys = y' + y'(jik,bac) + y'(kji,cba)
      // (D' is invariant too, so ys is formed from grad(t3') in one pass)
      const int ys = E.node(s6, false, false);
      if (pair) E.exec_sym6_div_adjoint_pair(-1.0, T3, es, E.v(Z), E.v(ys));
      else E.exec_sym3_div(T3, true, es, E.v(ys));
      const int Dv = E.node({v, v}), Do = E.node({o, o});
      // the two slot densities read the same tensors and write their own:
      // as parallel branches (the vv one FP32-bound, the oo one HBM-bound)
      E.branch_begin();
      E.exec_contract("ijkabc,ljkabc->li", 1.0, E.v(ys), false, T3, false, E.v(Do), false);
      E.branch_switch();
      E.exec_contract("ijkabc,ijkdbc->ad", 1.0, E.v(ys), false, T3, false, E.v(Dv), false);
      E.branch_join();
      const int tv = E.node({v, v}), to = E.node({o, o});
      E.exec_contract("Aa,AD->aD", 1.0, SIV, false, E.v(Dv), false, E.v(tv), false);
      E.exec_contract("aD,dD->ad", -1.0, E.v(tv), false, SV, false, wvv, true);
      E.exec_contract("lL,LI->lI", 1.0, SO, false, E.v(Do), false, E.v(to), false);
      E.exec_contract("lI,Ii->li", 1.0, E.v(to), false, SIO, false, woo, true);
    }, true);
  }
  // ---- X1, X2 in the rotated basis ------------------------------------------------
  const View T3 = E.v(t3p);
  // t - t(cba), 2 t^cbe - t^ceb - t^ebc and 2 t^cba - t^bca - t^abc from one
  // pass over t3' (four distinct permuted views)
  const int dd = E.node(s6, false, false);
  const int Ub = E.node(s6, false, false);
  const int Uc = E.node(s6, false, false);
  E.combine_multi({{{1.0, T3}, {-1.0, E.ev("ijkcba->ijkabc", T3)}},
                   {{2.0, T3}, {-1.0, E.ev("ijkxzy->ijkxyz", T3)}, {-1.0, E.ev("ijkzyx->ijkxyz", T3)}},
                   {{2.0, T3}, {-1.0, E.ev("mjkyxz->mjkxyz", T3)}, {-1.0, E.ev("mjkzyx->mjkxyz", T3)}}},
                  {E.v(dd), E.v(Ub), E.v(Uc)});
  // X1 = sum dd Lp (Eq. A21) and the first term of X2, S3 = sum dd Fp
  // (Eq. A22), as one operation whose reverse writes grad(dd) =
  // gX1 x Lp + gS3 x Fp in one pass (as two products, the second outer
  // product re-reads the first one's output)
  E.exec_contract_at("ijkabc,jkbc->ia", 1.0, E.v(dd), false, 0, Lp, false, 0, E.v(X1p), false, 0,
                     false);
  E.exec_contract_at("ijkabc,kc->ijab", 1.0, E.v(dd), false, 0, Fp, false, 0, E.v(S3p), false, 0,
                     false);
  {
    const bool gd = E.needs_grad(dd), gl = E.needs_grad(Lp.node), gf = E.needs_grad(Fp.node);
    if (gd || gl) E.set_needs_grad(X1p, true);
    if (gd || gf) E.set_needs_grad(S3p, true);
    if (gd || gl || gf)
      E.custom([&E, dd, Lp, Fp, X1p, S3p, gd, gl, gf]() {
        const bool hx = E.grad_ready(X1p), hs = E.grad_ready(S3p);
        if (gd)
          E.exec_outer_pair(hx ? 1.0 : 0.0, E.v(X1p), Lp, hs ? 1.0 : 0.0, E.v(S3p), Fp, E.v(dd));
        if (gl) E.exec_contract("ijkabc,ia->jkbc", 1.0, E.v(dd), false, E.v(X1p), true, Lp, true);
        if (gf) E.exec_contract("ijkabc,ijab->kc", 1.0, E.v(dd), false, E.v(S3p), true, Fp, true);
      }, true);
  }
  E.contract("ijkcbe,acke->ijab", 1.0, E.v(Ub), Gb, E.v(S3p), true);
  E.contract("mjkcba,kimc->ijab", -1.0, E.v(Uc), Gc, E.v(S3p), true);
  }
  // ---- rotate the results back: X = (S_o x S_v) X' -----------------------------
  const View X1t = rot("iI,IA->iA", SO, E.v(X1p), {o, v});
  E.contract("aA,iA->ia", 1.0, SV, X1t, R1, true);
  View S3 = rot("iI,IJAB->iJAB", SO, E.v(S3p), {o, o, v, v});
  S3 = rot("jJ,iJAB->ijAB", SO, S3, {o, o, v, v});
  S3 = rot("aA,ijAB->ijaB", SV, S3, {o, o, v, v});
  E.contract("bB,ijaB->ijab", 1.0, SV, S3, SD, true);
  return t3p;
}

// A t3 = rhs with A = eps3 + [V~, .] (Eq. 4 / Eq. A12 with dt3/dt = 0): +v~_ad on
// each virtual slot, -v~_li on each occupied slot.  Forward: `sweeps`
// fixed-point corrections t3 <- (rhs - S t3) / eps3 after t3 = rhs / eps3
// (the paper's iterative scheme on the stored tensor, Section 2.1).  Adjoint
// (implicit, no unrolled sweeps): y = A^-T grad(t3) by the same fixed point
// with S^T, then grad(rhs) += y, grad(v~_vv)[a,d] -= sum_slots y[..a..] t3[..d..]
// and grad(v~_oo)[l,i] += sum_slots y[i..] t3[l..] -- the triples terms of
// the one-electron density (the paper's D_ab and D_ij, Eqs. A31-A32).
template <typename R>
int field_coupled_solve(Engine<R>& E, int rhs, const View& wvv, const View& woo, int wt,
                        const typename Engine<R>::EpsSpec& es, const std::vector<int>& s6,
                        int sweeps) {
  const int t3 = E.node(s6, false, false);
  const int sx = E.node(s6, false, false);
  const View T3 = E.v(t3), SX = E.v(sx), RHS = E.v(rhs);
  // captures by value: the closure also runs later, in the reverse sweep
  auto apply = [&E, sx, wvv, woo](const View& src, bool src_grad, const View& x, bool transpose) {
    // SX = src - S x (S^T when transpose), on data buffers
    const View SX = E.v(sx);
    E.exec_copy(src, src_grad, SX);
    if (!transpose) {
      E.exec_contract("ad,ijkdbc->ijkabc", -1.0, wvv, false, x, false, SX, false);
      E.exec_contract("bd,ijkadc->ijkabc", -1.0, wvv, false, x, false, SX, false);
      E.exec_contract("cd,ijkabd->ijkabc", -1.0, wvv, false, x, false, SX, false);
      E.exec_contract("li,ljkabc->ijkabc", 1.0, woo, false, x, false, SX, false);
      E.exec_contract("lj,ilkabc->ijkabc", 1.0, woo, false, x, false, SX, false);
      E.exec_contract("lk,ijlabc->ijkabc", 1.0, woo, false, x, false, SX, false);
    } else {
      E.exec_contract("ad,ijkabc->ijkdbc", -1.0, wvv, false, x, false, SX, false);
      E.exec_contract("bd,ijkabc->ijkadc", -1.0, wvv, false, x, false, SX, false);
      E.exec_contract("cd,ijkabc->ijkabd", -1.0, wvv, false, x, false, SX, false);
      E.exec_contract("li,ijkabc->ljkabc", 1.0, woo, false, x, false, SX, false);
      E.exec_contract("lj,ijkabc->ilkabc", 1.0, woo, false, x, false, SX, false);
      E.exec_contract("lk,ijkabc->ijlabc", 1.0, woo, false, x, false, SX, false);
    }
  };
  E.exec_div(RHS, false, es, T3, false, true);
  for (int it = 0; it < sweeps; ++it) {
    apply(RHS, false, T3, false);
    E.exec_div(SX, false, es, T3, false, true);
  }
  const bool g = E.needs_grad(rhs) || E.needs_grad(wt);
  E.set_needs_grad(t3, g);
  if (g) {
    E.custom([&E, rhs, wt, t3, sx, wvv, woo, es, s6, sweeps, apply]() mutable {
      if (!E.needs_grad(t3)) return;
      const View T3 = E.v(t3), SX = E.v(sx);
      const int y = E.node(s6, false, false);
      const View Y = E.v(y);
      E.exec_div(T3, true, es, Y, false, true);  // y = grad(t3) / eps3
      for (int it = 0; it < sweeps; ++it) {
        apply(T3, true, Y, true);
        E.exec_div(SX, false, es, Y, false, true);
      }
      if (E.needs_grad(rhs)) E.exec_axpy(1.0, Y, false, E.v(rhs), true);
      if (E.needs_grad(wt)) {
        // t3 is invariant under the simultaneous permutations, so the slot-2
        // and slot-3 densities of y equal the slot-1 densities of the
        // permuted y: fold them into ys = y + y(jik,bac) + y(kji,cba)
        const int ys = E.node(s6, false, false);
        E.exec_combine({{1.0, Y}, {1.0, E.ev("jikbac->ijkabc", Y)}, {1.0, E.ev("kjicba->ijkabc", Y)}},
                       E.v(ys), true);
        const View YS = E.v(ys);
        E.exec_contract("ijkabc,ijkdbc->ad", -1.0, YS, false, T3, false, wvv, true);
        E.exec_contract("ijkabc,ljkabc->li", 1.0, YS, false, T3, false, woo, true);
      }
    }, true);
  }
  return t3;
}

template <typename R, typename Fill>
StageNodes record_stage(Engine<R>& E, const Hamil<R>& H, const StageOptions& opt, Fill&& fill) {
  const int o = H.o, v = H.v, n = H.n, na = H.naux;
  StageNodes S;
  S.t1 = E.node({o, v}, opt.need_grad);
  S.t2 = E.node({o, o, v, v}, opt.need_grad);
  S.w = E.node({n, n}, opt.need_grad);
  fill(S);
  // contractions recorded while the region is open (and their adjoints) may
  // take the tensor-core route
  const bool all_tc = opt.tc_scope >= 2 && E.tensor_cores() == 4;
  E.set_tc_region(all_tc);

  const int Lc = E.external(H.L, {na, n, n});
  const int hc = E.external(H.h, {n, n});
  const int on = E.external(H.ones, {n});
  const View ones_o = E.v(on).sub(0, 0, o);
  const View T = E.v(S.t2);

  // ---- T1 dressing: X = 1 - tau, Y = 1 + tau, tau[a,i] = t_i^a ----------------
  const int X = E.node({n, n}), Y = E.node({n, n});
  E.fill_identity(X);
  E.fill_identity(Y);
  const View t1T = E.ev("ia->ai", E.v(S.t1));
  E.axpy(-1.0, t1T, E.v(X).sub(0, o, v).sub(1, 0, o));
  E.axpy(1.0, t1T, E.v(Y).sub(0, o, v).sub(1, 0, o));
  const int LX = E.node({na, n, n}, false, false), Lt = E.node({na, n, n}, false, false);
  E.contract("pr,Prs->Pps", 1.0, E.v(X), E.v(Lc), E.v(LX), false);
  E.contract("Pps,sq->Ppq", 1.0, E.v(LX), E.v(Y), E.v(Lt), false);
  const int hw = E.node({n, n}), hX = E.node({n, n}, false, false), ht = E.node({n, n}, false, false);
  E.axpy(1.0, E.v(hc), E.v(hw));
  E.axpy(1.0, E.v(S.w), E.v(hw));
  E.contract("pr,rs->ps", 1.0, E.v(X), E.v(hw), E.v(hX), false);
  E.contract("ps,sq->pq", 1.0, E.v(hX), E.v(Y), E.v(ht), false);
  const int wX = E.node({n, n}, false, false), wt = E.node({n, n}, false, false);
  E.contract("pr,rs->ps", 1.0, E.v(X), E.v(S.w), E.v(wX), false);
  E.contract("ps,sq->pq", 1.0, E.v(wX), E.v(Y), E.v(wt), false);
  // the field-dressed eigenbasis only needs w~: start it now, beside the CCSD part
  FieldBasis<R> fb;
  if (opt.triples && opt.field_terms && opt.rotation) fb = start_field_basis(E, H, wt, opt.basis);
  const int g = E.node({n, n, n, n}, false, false);
  E.set_tc_region(all_tc || (opt.tc_scope >= 1 && E.tensor_cores() == 4));
  E.contract("Ppq,Prs->pqrs", 1.0, E.v(Lt), E.v(Lt), E.v(g), false);
  E.set_tc_region(all_tc);
  // f~ = h~ + sum_k 2 g~_pqkk - g~_pkkq
  const int ft = E.node({n, n});
  E.axpy(1.0, E.v(ht), E.v(ft));
  E.contract("pqk,k->pq", 2.0, E.ev("pqkk->pqk", E.v(g).sub(2, 0, o).sub(3, 0, o)), ones_o,
             E.v(ft), true);
  E.contract("pkq,k->pq", -1.0, E.ev("pkkq->pkq", E.v(g).sub(1, 0, o).sub(2, 0, o)), ones_o,
             E.v(ft), true);

  // block views: 'o' -> [0,o), 'v' -> [o,n)
  auto blk = [&](int node, const char* b) {
    View r = E.v(node);
    for (int d = 0; b[d]; ++d) r = (b[d] == 'o') ? r.sub(d, 0, o) : r.sub(d, o, v);
    return r;
  };
  auto G = [&](const char* b) { return blk(g, b); };
  auto F = [&](const char* b) { return blk(ft, b); };

  // ---- CCSD residual (T1-transformed, spin adapted) ---------------------------
  S.r1 = E.node({o, v});
  const View R1 = E.v(S.r1);
  S.r2 = E.node({o, o, v, v});
  const View R2 = E.v(S.r2);
  const int Sd = E.node({o, o, v, v});
  const View SD = E.v(Sd);
  const int Lov = E.node({o, v, o, v}, false, false);
  E.combine({{2.0, G("ovov")}, {-1.0, E.ev("lckd->ldkc", G("ovov"))}}, E.v(Lov), true);
  // With the triples beside it, the CCSD part runs as a concurrent region of
  // the stage (and of its reverse pass): it reads private copies of the
  // dressed integrals, f~ and t2 and writes R1c, SDc, added to R1, SD after
  // the join, so no value or cotangent is written from both sides.
  const bool region = opt.ccsd && opt.triples && !all_tc && E.regions();
  int gq = g, fq = ft, R1n = S.r1, SDn = Sd;
  View Tq = T;
  if (region) {
    gq = E.node({n, n, n, n}, false, false);
    E.combine({{1.0, E.v(g)}}, E.v(gq), true);
    fq = E.node({n, n}, false, false);
    E.combine({{1.0, E.v(ft)}}, E.v(fq), true);
    const int tq = E.node({o, o, v, v}, false, false);
    E.combine({{1.0, T}}, E.v(tq), true);
    Tq = E.v(tq);
    E.region_begin();
    R1n = E.node({o, v});
    SDn = E.node({o, o, v, v});
  }
  if (opt.ccsd) {
  auto Gq = [&](const char* b) { return blk(gq, b); };
  auto Fq = [&](const char* b) { return blk(fq, b); };
  const View R1q = E.v(R1n), SDq = E.v(SDn);
  const int u = E.node({o, o, v, v}, false, false);
  E.combine({{2.0, Tq}, {-1.0, E.ev("ijba->ijab", Tq)}}, E.v(u), true);
  const View U = E.v(u);
  int Lq = Lov;
  if (region) {
    Lq = E.node({o, v, o, v}, false, false);
    E.combine({{2.0, Gq("ovov")}, {-1.0, E.ev("lckd->ldkc", Gq("ovov"))}}, E.v(Lq), true);
  }
  E.contract("kicd,adkc->ia", 1.0, U, Gq("vvov"), R1q, true);
  E.contract("klac,kilc->ia", -1.0, U, Gq("ooov"), R1q, true);
  E.contract("ikac,kc->ia", 1.0, U, Fq("ov"), R1q, true);
  E.axpy(1.0, E.ev("ai->ia", Fq("vo")), R1q);

  E.axpy(1.0, E.ev("aibj->ijab", Gq("vovo")), R2);
  E.contract("ijcd,acbd->ijab", 1.0, Tq, Gq("vvvv"), R2, true);
  const int Wk = E.node({o, o, o, o});
  E.axpy(1.0, Gq("oooo"), E.v(Wk));
  E.contract("ijcd,kcld->kilj", 1.0, Tq, Gq("ovov"), E.v(Wk), true);
  E.contract("klab,kilj->ijab", 1.0, Tq, E.v(Wk), R2, true);
  const int Xc = E.node({o, o, v, v});
  E.axpy(1.0, Gq("oovv"), E.v(Xc));
  E.contract("liad,kdlc->kiac", -0.5, Tq, Gq("ovov"), E.v(Xc), true);
  E.contract("kjbc,kiac->ijab", -0.5, Tq, E.v(Xc), SDq, true);
  E.contract("kibc,kjac->ijab", -1.0, Tq, E.v(Xc), SDq, true);
  const int Ltv = E.node({v, o, o, v});
  E.axpy(2.0, Gq("voov"), E.v(Ltv));
  E.axpy(-1.0, E.ev("acki->aikc", Gq("vvoo")), E.v(Ltv));
  const int Xd = E.node({o, v, o, v});
  E.axpy(1.0, E.ev("aikc->iakc", E.v(Ltv)), E.v(Xd));
  E.contract("ilad,ldkc->iakc", 0.5, U, E.v(Lq), E.v(Xd), true);
  E.contract("jkbc,iakc->ijab", 0.5, U, E.v(Xd), SDq, true);
  const int Fvv = E.node({v, v}), Foo = E.node({o, o});
  E.axpy(1.0, Fq("vv"), E.v(Fvv));
  E.contract("klbd,ldkc->bc", -1.0, U, Gq("ovov"), E.v(Fvv), true);
  E.axpy(1.0, Fq("oo"), E.v(Foo));
  E.contract("ljcd,kdlc->kj", 1.0, U, Gq("ovov"), E.v(Foo), true);
  E.contract("ijac,bc->ijab", 1.0, Tq, E.v(Fvv), SDq, true);
  E.contract("ikab,kj->ijab", -1.0, Tq, E.v(Foo), SDq, true);
  }  // opt.ccsd
  E.region_end();

  // ---- triples ---------------------------------------------------------------
  if (opt.triples && opt.field_terms && opt.rotation) {
    E.set_tc_region(true);  // the dense triples contractions may use tensor cores
    S.t3 = rotated_triples(E, H, T, wt, fb, g, ft, R1, SD, blk, opt.triples_chunk);
    E.set_tc_region(all_tc);
  } else if (opt.triples) {
    E.set_tc_region(true);  // the dense triples contractions may use tensor cores
    const std::vector<int> s6 = {o, o, o, v, v, v};
    const bool field = opt.field_terms;
    if (!field && opt.triples_chunk > 0) {
      // field-free and blocked: W and t3 per slab, never stored
      typename Engine<R>::EpsSpec es;
      es.o = o;
      es.v = v;
      es.osum_r = H.osum_r;
      es.vsum_r = H.vsum_r;
      const int Ljk = E.node({o, o, v, v}, false, false);
      E.combine({{2.0, E.ev("jbkc->jkbc", G("ovov"))}, {-1.0, E.ev("jckb->jkbc", G("ovov"))}},
                E.v(Ljk), true);
      const int X1o = E.node({o, v}), S3o = E.node({o, o, v, v});
      blocked_triples<R>(E, o, v, opt.triples_chunk,
                         {T, E.ev("ckbe->ekbc", G("vovv")), T, G("oovo"), E.v(Ljk), F("ov"),
                          G("vvov"), G("ooov")},
                         es, X1o, S3o, FieldAdjoint());
      E.axpy(1.0, E.v(X1o), R1);
      E.axpy(1.0, E.v(S3o), SD);
    } else {
      // Z = sum_e t_ij^ae <cb|ke>~ - sum_m t_im^ab <mc|jk>~ ; W = P_ijk^abc Z (Eqs. A25, A30)
      const int Z = E.node(s6, false, false);
      E.contract("ijae,ckbe->ijkabc", 1.0, T, G("vovv"), E.v(Z), false);
      E.contract("imab,mjck->ijkabc", -1.0, T, G("oovo"), E.v(Z), true);
      // rhs = -(W + <mu3|1/2[[V~,T2],T2]|0>), the latter = -P sum_ld v~_ld t_ij^ad t_kl^cb:
      // P is linear, so the source is folded into Z and rhs = -P(Z)
      if (field) {
        const int Yl = E.node({o, o, o, v}, false, false);
        E.contract("ld,ijad->lija", 1.0, blk(wt, "ov"), T, E.v(Yl), false);
        E.contract("lija,klcb->ijkabc", -1.0, E.v(Yl), T, E.v(Z), true);
      }
      typename Engine<R>::EpsSpec es;
      es.eps = H.eps;
      for (int d = 0; d < 3; ++d) { es.sign[d] = -1; es.base[d] = 0; }
      for (int d = 3; d < 6; ++d) { es.sign[d] = 1; es.base[d] = o; }
      es.osum = H.osum;
      es.vsum = H.vsum;
      es.osum_r = H.osum_r;
      es.vsum_r = H.vsum_r;
      es.order = H.orbit_order;
      es.o = o;
      es.v = v;
      int t3;
      if (!field) {
        t3 = E.node(s6, false, false);
        E.sym6_div(-1.0, E.v(Z), es, E.v(t3));
      } else {
        const int rhs = E.node(s6, false, false);
        E.sym6(-1.0, E.v(Z), E.v(rhs), true);
        t3 = field_coupled_solve(E, rhs, blk(wt, "vv"), blk(wt, "oo"), wt, es, s6,
                                 std::max(1, opt.field_iters));
      }
      S.t3 = t3;
      const View T3 = E.v(t3);
      // X1 (Eq. A21) and X2 (Eq. A22)
      const int dd = E.node(s6, false, false);  // t_ijk^abc - t_ijk^cba
      const int Ub = E.node(s6, false, false);  // 2 t^cbe - t^ceb - t^ebc  as [ijk cbe]
      const int Uc = E.node(s6, false, false);  // 2 t_mjk^cba - t_mjk^bca - t_mjk^abc
      E.combine_multi({{{1.0, T3}, {-1.0, E.ev("ijkcba->ijkabc", T3)}},
                       {{2.0, T3}, {-1.0, E.ev("ijkxzy->ijkxyz", T3)}, {-1.0, E.ev("ijkzyx->ijkxyz", T3)}},
                       {{2.0, T3}, {-1.0, E.ev("mjkyxz->mjkxyz", T3)}, {-1.0, E.ev("mjkzyx->mjkxyz", T3)}}},
                      {E.v(dd), E.v(Ub), E.v(Uc)});
      const int Ljk = E.node({o, o, v, v}, false, false);
      E.combine({{2.0, E.ev("jbkc->jkbc", G("ovov"))}, {-1.0, E.ev("jckb->jkbc", G("ovov"))}},
                E.v(Ljk), true);
      E.contract("ijkabc,jkbc->ia", 1.0, E.v(dd), E.v(Ljk), R1, true);
      const int S3 = E.node({o, o, v, v}, false, false);
      E.contract("ijkabc,kc->ijab", 1.0, E.v(dd), F("ov"), E.v(S3), false);
      E.contract("ijkcbe,acke->ijab", 1.0, E.v(Ub), G("vvov"), E.v(S3), true);
      E.contract("mjkcba,kimc->ijab", -1.0, E.v(Uc), G("ooov"), E.v(S3), true);
      E.axpy(1.0, E.v(S3), SD);
    }
    E.set_tc_region(all_tc);
  }
  if (region) {
    E.region_join();
    E.axpy(1.0, E.v(R1n), R1);
    E.axpy(1.0, E.v(SDn), SD);
  }
  // P_ij^ab on the symmetrised part
  E.combine({{1.0, SD}, {1.0, E.ev("jiba->ijab", SD)}}, R2, false);

  // ---- energy <0|H + [H,T2]|0> - E_ref (Eq. A8) --------------------------------
  // With canonical orbitals (F_ia = 0) the dressed expression equals
  //   2 sum_i w_ii + 2 sum_ia w_ia t_i^a + sum_iajb L_iajb (t_ij^ab + t_i^a t_j^b),
  // L_iajb = 2 g_iajb - g_ibja (the ov|ov block is not changed by the
  // dressing). The graph holds the last sum only, so no reference-sized term
  // is summed in the compute precision; the field terms (and their t1 and w
  // derivatives) are added in FP64 by the integrator kernels.
  S.e = E.node({});
  const View Ev = E.v(S.e);
  const int tL = E.node({o, v}, false, false);
  E.contract("ia,iajb->jb", 1.0, E.v(S.t1), E.v(Lov), E.v(tL), false);
  E.contract("jb,jb->", 1.0, E.v(tL), E.v(S.t1), Ev, true);
  E.contract("ijab,iajb->", 1.0, T, E.v(Lov), Ev, true);
  E.set_tc_region(false);
  return S;
}

}  // namespace rtcc3
