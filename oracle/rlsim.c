/*
 * CPU oracle for the rigid-sphere task bodies -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain C99, single precision, one IEEE rounding per written operation:
 * build with -ffp-contract=off (no fused multiply-add) and no fast-math.
 * Division and sqrtf are correctly rounded. Loops run in the order stated,
 * which defines the results bit for bit.
 *
 * This workload stands in for the paper's Brax physics environments (Sec. II,
 * "Case Study 1": many small kernels per step, contact sets that depend on the
 * simulated state, so the task graph changes with the input). The paper prints
 * no physics, so the bodies below are this workload's definition:
 *
 *   broadphase  for every sphere pair i < j (lexicographic), contact iff
 *               ((dx*dx + dy*dy) + dz*dz) < (r_i + r_j)^2, d = p_j - p_i;
 *               islands = connected components of the contact graph, each
 *               labelled by its smallest sphere index; an island counts when
 *               it has at least one contact.
 *   solve       8 Gauss-Seidel sweeps over the contacts in list order; per
 *               contact a non-negative normal impulse
 *               dl = (beta_dt * max(pen - slop, 0) - v_n) / (w_i + w_j).
 *   integrate   semi-implicit Euler (v_z += g dt; p += v dt) and walls of a
 *               cubic box [r, L - r] that clamp p and reflect v with factor 1/2.
 *
 * Parity: pinned by closed forms and invariants in tests/test_oracle_bodies.py
 * (free fall, a symmetric head-on pair, momentum of an isolated island,
 * brute-force fp64 distances, connected components by graph search).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define NSPH 32
#define NPAIR (NSPH * (NSPH - 1) / 2)
#define REC_BYTES 1088
#define SWEEPS 8

typedef struct {
    uint32_t ncontact;
    uint32_t nisland;
    uint8_t label[NSPH];
    uint8_t root[NSPH];
    uint16_t pair[NPAIR];      /* i | (j << 8), i < j */
    uint8_t pad[REC_BYTES - 8 - 2 * NSPH - 2 * NPAIR];
} contact_rec;

typedef char rec_size_check[(sizeof(contact_rec) == REC_BYTES) ? 1 : -1];

void oracle_rl_broadphase(const float *pos, const float *prop, uint8_t *cont,
                          uint32_t *nisl, uint32_t nenv)
{
    for (uint32_t e = 0; e < nenv; ++e) {
        const float *p = pos + (size_t)e * NSPH * 3;
        const float *pr = prop + (size_t)e * NSPH * 2;
        contact_rec rec;
        memset(&rec, 0, sizeof rec);
        uint32_t nc = 0;
        for (int i = 0; i < NSPH; ++i) {
            for (int j = i + 1; j < NSPH; ++j) {
                float dx = p[j * 3 + 0] - p[i * 3 + 0];
                float dy = p[j * 3 + 1] - p[i * 3 + 1];
                float dz = p[j * 3 + 2] - p[i * 3 + 2];
                float xx = dx * dx;
                float yy = dy * dy;
                float zz = dz * dz;
                float d2 = xx + yy;
                d2 = d2 + zz;
                float rs = pr[i * 2] + pr[j * 2];
                float rs2 = rs * rs;
                if (d2 < rs2)
                    rec.pair[nc++] = (uint16_t)(i | (j << 8));
            }
        }
        rec.ncontact = nc;
        /* connected components: relax label = min(label) over contacts until fixed */
        int lab[NSPH], deg[NSPH];
        for (int i = 0; i < NSPH; ++i) { lab[i] = i; deg[i] = 0; }
        for (uint32_t k = 0; k < nc; ++k) {
            deg[rec.pair[k] & 255]++;
            deg[rec.pair[k] >> 8]++;
        }
        int changed = 1;
        while (changed) {
            changed = 0;
            for (uint32_t k = 0; k < nc; ++k) {
                int i = rec.pair[k] & 255, j = rec.pair[k] >> 8;
                int m = lab[i] < lab[j] ? lab[i] : lab[j];
                if (lab[i] != m) { lab[i] = m; changed = 1; }
                if (lab[j] != m) { lab[j] = m; changed = 1; }
            }
        }
        uint32_t ni = 0;
        for (int i = 0; i < NSPH; ++i) {
            rec.label[i] = (uint8_t)lab[i];
            if (lab[i] == i && deg[i] > 0)
                rec.root[ni++] = (uint8_t)i;
        }
        rec.nisland = ni;
        memcpy(cont + (size_t)e * REC_BYTES, &rec, REC_BYTES);
        nisl[e] = ni;
    }
}

void oracle_rl_solve(const float *pos, const float *prop, const uint8_t *cont,
                     float *vel, float beta_dt, float slop)
{
    contact_rec rec;
    memcpy(&rec, cont, REC_BYTES);
    for (int it = 0; it < SWEEPS; ++it) {
        for (uint32_t k = 0; k < rec.ncontact; ++k) {
            int i = rec.pair[k] & 255, j = rec.pair[k] >> 8;
            const float *pi = pos + i * 3, *pj = pos + j * 3;
            float *vi = vel + i * 3, *vj = vel + j * 3;
            float dx = pj[0] - pi[0];
            float dy = pj[1] - pi[1];
            float dz = pj[2] - pi[2];
            float xx = dx * dx;
            float yy = dy * dy;
            float zz = dz * dz;
            float d2 = xx + yy;
            d2 = d2 + zz;
            float dist = sqrtf(d2);
            float nx, ny, nz;
            if (dist > 0.0f) {
                nx = dx / dist;
                ny = dy / dist;
                nz = dz / dist;
            } else {
                nx = 0.0f; ny = 0.0f; nz = 1.0f;
            }
            float rsum = prop[i * 2] + prop[j * 2];
            float pen = rsum - dist;
            float dvx = vj[0] - vi[0];
            float dvy = vj[1] - vi[1];
            float dvz = vj[2] - vi[2];
            float tx = dvx * nx;
            float ty = dvy * ny;
            float tz = dvz * nz;
            float vn = tx + ty;
            vn = vn + tz;
            float excess = pen - slop;
            if (!(excess > 0.0f))
                excess = 0.0f;
            float bias = beta_dt * excess;
            float wsum = prop[i * 2 + 1] + prop[j * 2 + 1];
            float num = bias - vn;
            float dl = num / wsum;
            if (dl > 0.0f) {
                float ai = dl * prop[i * 2 + 1];
                float aj = dl * prop[j * 2 + 1];
                float q;
                q = ai * nx; vi[0] = vi[0] - q;
                q = ai * ny; vi[1] = vi[1] - q;
                q = ai * nz; vi[2] = vi[2] - q;
                q = aj * nx; vj[0] = vj[0] + q;
                q = aj * ny; vj[1] = vj[1] + q;
                q = aj * nz; vj[2] = vj[2] + q;
            }
        }
    }
}

void oracle_rl_integrate(float *pos, float *vel, const float *prop, uint32_t nenv,
                         float dt, float gdt, float box)
{
    for (uint32_t s = 0; s < nenv * NSPH; ++s) {
        float *p = pos + (size_t)s * 3, *v = vel + (size_t)s * 3;
        float r = prop[(size_t)s * 2];
        float lo = r;
        float hi = box - r;
        v[2] = v[2] + gdt;
        for (int a = 0; a < 3; ++a) {
            float step = v[a] * dt;
            p[a] = p[a] + step;
            if (p[a] < lo) {
                p[a] = lo;
                if (v[a] < 0.0f) v[a] = v[a] * -0.5f;
            } else if (p[a] > hi) {
                p[a] = hi;
                if (v[a] > 0.0f) v[a] = v[a] * -0.5f;
            }
        }
    }
}
