// The sub-elements that replace a split element (Sec. 3), as one function for
// host and device: the CUDA path runs it in k_create_subs, the host tests
// compile it with g++ and compare it with the oracle's rule, and a device probe
// (cem_probe_split_rule) runs it on the GPU for the same comparison.
//
// Pattern I (two local nodes per side, P = {p0, p1} with side bit 0 and
// Q = {q0, q1} with bit 1, each ascending): two triangular prisms, first
// (p0, M(p0,q0), M(p0,q1)) over (p1, M(p1,q0), M(p1,q1)), then
// (q0, M(q0,p0), M(q0,p1)) over (q1, M(q1,p0), M(q1,p1)).
// Pattern II (one local node c cut off, o0 < o1 < o2 the others): the corner
// tetrahedron (c, M(c,o0), M(c,o1), M(c,o2)), then the prism
// (M(o0,c), M(o1,c), M(o2,c)) over (o0, o1, o2).
// M(x, y) is the new node on the element's edge x-y that stays attached to x.
//
// A prism A0 A1 A2 / B0 B1 B2 (rails Ai - Bi) is divided into three
// tetrahedra (the remainder rule of Sec. 3).  Each quadrilateral face is cut
// along the diagonal through its vertex with the smallest creation id, so two
// elements sharing a quadrilateral (neighbours split by the same crack) cut it
// alike and the sub-element mesh stays conforming.  With the prism turned so
// that its smallest vertex is v1 (v1 v2 v3 one triangle, v4 v5 v6 the other,
// rails v1-v4, v2-v5, v3-v6), the faces through v1 take the diagonals v1-v5
// and v1-v6, and the face v2 v3 v6 v5 takes v2-v6 when min(v2, v6) <
// min(v3, v5), else v3-v5; each case has one division into three tetrahedra.
// Orientation is left to the caller.
//
// Everything is written with scalars and selects: no local array is indexed
// by a run-time value and no pointer chooses between local arrays, so the
// device code keeps the whole rule in registers.  (A first device version
// that selected between the two triangles' local arrays through a pointer
// produced wrong sub-elements on sm_103a while the same source compiled for
// the host was right.)
#pragma once

#ifndef __CUDACC__
#define CEM_HD inline
#else
#define CEM_HD __host__ __device__ __forceinline__
#endif

// x_j for j in {0, 1, 2} / {0, 1, 2, 3}, by selects
CEM_HD int cem_pick3(int x0, int x1, int x2, int j) { return j == 0 ? x0 : (j == 1 ? x1 : x2); }
CEM_HD int cem_pick4(int x0, int x1, int x2, int x3, int j) {
    return j == 0 ? x0 : (j == 1 ? x1 : (j == 2 ? x2 : x3));
}

// The three tetrahedra of prism (a0 a1 a2 / b0 b1 b2), vertex creation ids
// ea* / eb*, written to out[r0 .. r0+2][0..3] (r0 a compile-time row after
// inlining).
CEM_HD void cem_prism_division6(int a0, int a1, int a2, int b0, int b1, int b2, int ea0, int ea1, int ea2, int eb0,
                                int eb1, int eb2, int out[][4], int r0) {
    // the smallest id: its triangle (0: a, 1: b) and corner j; ties to the first in a0..b2 order
    int tri = 0, j = 0, best = ea0;
    if (ea1 < best) { best = ea1; j = 1; }
    if (ea2 < best) { best = ea2; j = 2; }
    if (eb0 < best) { best = eb0; tri = 1; j = 0; }
    if (eb1 < best) { best = eb1; tri = 1; j = 1; }
    if (eb2 < best) { best = eb2; tri = 1; j = 2; }
    const int j1 = j == 2 ? 0 : j + 1, j2 = j == 0 ? 2 : j - 1;
    const int l0 = tri ? b0 : a0, l1 = tri ? b1 : a1, l2 = tri ? b2 : a2;
    const int h0 = tri ? a0 : b0, h1 = tri ? a1 : b1, h2 = tri ? a2 : b2;
    const int le0 = tri ? eb0 : ea0, le1 = tri ? eb1 : ea1, le2 = tri ? eb2 : ea2;
    const int he0 = tri ? ea0 : eb0, he1 = tri ? ea1 : eb1, he2 = tri ? ea2 : eb2;
    const int v1 = cem_pick3(l0, l1, l2, j), v2 = cem_pick3(l0, l1, l2, j1), v3 = cem_pick3(l0, l1, l2, j2);
    const int v4 = cem_pick3(h0, h1, h2, j), v5 = cem_pick3(h0, h1, h2, j1), v6 = cem_pick3(h0, h1, h2, j2);
    const int e2 = cem_pick3(le0, le1, le2, j1), e3 = cem_pick3(le0, le1, le2, j2);
    const int e5 = cem_pick3(he0, he1, he2, j1), e6 = cem_pick3(he0, he1, he2, j2);
    const int m26 = e2 < e6 ? e2 : e6, m35 = e3 < e5 ? e3 : e5;
    const bool d26 = m26 < m35;   // the face v2 v3 v6 v5 is cut along v2-v6 (else v3-v5)
    out[r0][0] = v1;
    out[r0][1] = v2;
    out[r0][2] = v3;
    out[r0][3] = d26 ? v6 : v5;
    out[r0 + 1][0] = v1;
    out[r0 + 1][1] = d26 ? v2 : v5;
    out[r0 + 1][2] = d26 ? v6 : v3;
    out[r0 + 1][3] = d26 ? v5 : v6;
    out[r0 + 2][0] = v1;
    out[r0 + 2][1] = v5;
    out[r0 + 2][2] = v6;
    out[r0 + 2][3] = v4;
}

// The same division for vertices given as arrays (host tests).
CEM_HD void cem_prism_division(const int A[3], const int B[3], const int Ae[3], const int Be[3], int out[3][4]) {
    cem_prism_division6(A[0], A[1], A[2], B[0], B[1], B[2], Ae[0], Ae[1], Ae[2], Be[0], Be[1], Be[2], out, 0);
}

// Sub-elements of an element split with side mask m (bit l: side of local
// node l; 2 bits set is pattern I, 1 or 3 is pattern II).  n0..n3: the
// element's nodes, x0..x3 their creation ids.  mf(x, y, &node, &id): the new
// node on local edge x-y attached to x and its creation id.  Fills subs[0..k)
// in canonical order and returns k (6 or 4).
template <class MF>
CEM_HD int cem_split_subs(int n0, int n1, int n2, int n3, int x0, int x1, int x2, int x3, int m, const MF& mf,
                          int subs[6][4]) {
    int ones = 0;
    for (int l = 0; l < 4; ++l) ones += (m >> l) & 1;
    if (ones == 2) {
        int p0 = -1, p1 = -1, q0 = -1, q1 = -1;
        for (int l = 0; l < 4; ++l) {
            if ((m >> l) & 1) {
                if (q0 < 0) q0 = l;
                else q1 = l;
            } else {
                if (p0 < 0) p0 = l;
                else p1 = l;
            }
        }
        int g00, g01, g10, g11, e00, e01, e10, e11;
        // side of P: (p0, M(p0,q0), M(p0,q1)) over (p1, M(p1,q0), M(p1,q1))
        mf(p0, q0, &g00, &e00);
        mf(p0, q1, &g01, &e01);
        mf(p1, q0, &g10, &e10);
        mf(p1, q1, &g11, &e11);
        cem_prism_division6(cem_pick4(n0, n1, n2, n3, p0), g00, g01, cem_pick4(n0, n1, n2, n3, p1), g10, g11,
                            cem_pick4(x0, x1, x2, x3, p0), e00, e01, cem_pick4(x0, x1, x2, x3, p1), e10, e11, subs, 0);
        // side of Q: (q0, M(q0,p0), M(q0,p1)) over (q1, M(q1,p0), M(q1,p1))
        mf(q0, p0, &g00, &e00);
        mf(q0, p1, &g01, &e01);
        mf(q1, p0, &g10, &e10);
        mf(q1, p1, &g11, &e11);
        cem_prism_division6(cem_pick4(n0, n1, n2, n3, q0), g00, g01, cem_pick4(n0, n1, n2, n3, q1), g10, g11,
                            cem_pick4(x0, x1, x2, x3, q0), e00, e01, cem_pick4(x0, x1, x2, x3, q1), e10, e11, subs, 3);
        return 6;
    }
    // pattern II: the lone node c is the single node of its side
    int c = -1, first0 = -1;
    for (int l = 0; l < 4; ++l) {
        if ((m >> l) & 1) c = l;
        else if (first0 < 0) first0 = l;
    }
    if (ones != 1) c = first0;
    const int o0 = c == 0 ? 1 : 0, o1 = c <= 1 ? 2 : 1, o2 = c <= 2 ? 3 : 2;
    int k0, k1, k2, i0, i1, i2;
    mf(c, o0, &k0, &i0);
    mf(c, o1, &k1, &i1);
    mf(c, o2, &k2, &i2);
    subs[0][0] = cem_pick4(n0, n1, n2, n3, c);
    subs[0][1] = k0;
    subs[0][2] = k1;
    subs[0][3] = k2;
    mf(o0, c, &k0, &i0);
    mf(o1, c, &k1, &i1);
    mf(o2, c, &k2, &i2);
    cem_prism_division6(k0, k1, k2, cem_pick4(n0, n1, n2, n3, o0), cem_pick4(n0, n1, n2, n3, o1),
                        cem_pick4(n0, n1, n2, n3, o2), i0, i1, i2, cem_pick4(x0, x1, x2, x3, o0),
                        cem_pick4(x0, x1, x2, x3, o1), cem_pick4(x0, x1, x2, x3, o2), subs, 1);
    return 4;
}

#undef CEM_HD
