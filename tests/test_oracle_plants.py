"""Every plausible mistake planted in the oracle must trip at least one pin.

Each case copies dade_oracle.c, applies one textual change (a dropped term, a
wrong sign, an inverted ratio, a transposed operand, an off-by-one ...),
builds it on the CPU into a temporary directory and runs the pins against it.
The original file is never modified.
"""
import os
import tempfile

import pytest

import oracle
import pins

PLANTS = [
    ("estimate_ratio_inverted", "return Lam[D] / Lam[d] * Pd;", "return Lam[d] / Lam[D] * Pd;"),
    ("one_minus_eps", "double bound = (1.0 + eps[d]) * r;", "double bound = (1.0 - eps[d]) * r;"),
    ("eps_not_applied", "double bound = (1.0 + eps[d]) * r;", "double bound = r;"),
    ("reject_on_equality", "if (est > bound) { *dims = d; return 0; }",
     "if (est >= bound) { *dims = d; return 0; }"),
    ("strict_accept", "            return P <= r2;\n        }", "            return P < r2;\n        }"),
    ("rotation_transposed", "for (int k = 0; k < d; ++k) o[k] += w[k] * y;",
     "for (int k = 0; k < d; ++k) o[k] += W[(int64_t)k * d + j] * y;"),
    # E[X X^T] without the centring of Lemma 1 (both factors uncentred; one
    # uncentred factor alone is not a mistake since sum_i (x_ij - mu_j) = 0)
    ("covariance_not_centred", ["double yj = (double)x[j] - mu[j];", "row[k] += yj * ((double)x[k] - mu[k]);"],
     ["double yj = (double)x[j];", "row[k] += yj * ((double)x[k]);"]),
    ("eigen_ascending", "if (lam[j] > lam[best]) best = j;", "if (lam[j] < lam[best]) best = j;"),
    ("jacobi_sign", "double np = c * apk - s * aqk, nq = s * apk + c * aqk;",
     "double np = c * apk + s * aqk, nq = s * apk + c * aqk;"),
    ("quantile_floor", "(int64_t)ceil((1.0 - alpha) * (double)m);", "(int64_t)floor((1.0 - alpha) * (double)m);"),
    ("quantile_alpha_side", "(int64_t)ceil((1.0 - alpha) * (double)m);", "(int64_t)ceil(alpha * (double)m);"),
    ("rho_without_sqrt", "rho[(int64_t)t * m + kept] = sqrt(LD / Ld * Pd[dd - 1] / PD);",
     "rho[(int64_t)t * m + kept] = LD / Ld * Pd[dd - 1] / PD;"),
    ("rho_prefix_off_by_one", "for (int k = 0; k < dd; ++k) Ld += lam[k];",
     "for (int k = 0; k <= dd && k < d; ++k) Ld += lam[k];"),
    ("increment_drops_a_dim", "for (int k = d; k < dn; ++k) { double t = q[k] - o[k]; P += t * t; }",
     "for (int k = d; k < dn - 1; ++k) { double t = q[k] - o[k]; P += t * t; }"),
    ("heap_tie_reversed", "return (x->id > y->id) - (x->id < y->id);", "return (x->id < y->id) - (x->id > y->id);"),
    ("nearest_tie_high", "if (t < b1) { b2 = b1; b1 = t; best = c; }", "if (t <= b1) { b2 = b1; b1 = t; best = c; }"),
    ("empty_cluster_zeroed", "            if (cnt[c] > 0)\n                for (int k = 0; k < d; ++k) cent[(int64_t)c * d + k] = sum",
     "            if (cnt[c] >= 0)\n                for (int k = 0; k < d; ++k) cent[(int64_t)c * d + k] = sum"),
    ("threshold_not_refreshed", "double r2 = ntop == K ? buf[K - 1].key : INFINITY;", "double r2 = INFINITY;"),
    ("threshold_is_first_not_kth", "double r2 = ntop == K ? buf[K - 1].key : INFINITY;",
     "double r2 = ntop == K ? buf[0].key : INFINITY;"),
    ("seed_threshold_one_list_late", "if (seed > 0 && j == seed) r2_seed", "if (seed > 0 && j == seed + 1) r2_seed"),
    ("seed_threshold_not_frozen", "if (seed > 0 && j >= seed) r2 = r2_seed;", "if (seed > 0 && j > seed) r2 = r2_seed;"),
    # lagged tile schedule: r of tile t taken one tile late / written to the wrong ring slot
    ("lag_off_by_one", "epoch - 1 - lag >= 0 ? hist[(epoch - 1 - lag) % (lag + 1)]",
     "epoch - lag >= 0 ? hist[(epoch - lag) % (lag + 1)]"),
    ("lag_ring_index", "hist[epoch % (lag + 1)] = ", "hist[(epoch + 1) % (lag + 1)] = "),
    # row rounds: threshold never refreshed, rounds growing linearly, a row skipped per round
    ("rounds_threshold_not_refreshed", "double r2 = ntop < K ? INFINITY : buf[K - 1].key;", "double r2 = INFINITY;"),
    ("rounds_not_doubling", "hi = 2 * hi;", "hi = hi + tile;"),
    ("rounds_first_row_skipped", "for (int64_t t = lo; t < hi && t < len; ++t)",
     "for (int64_t t = lo + (lo > 0); t < hi && t < len; ++t)"),
    # the decision bracket moves the threshold the wrong way
    ("bias_sign", "double r2b = (r2_) * (1.0 + bias), d2", "double r2b = (r2_) * (1.0 - bias), d2"),
    # HNSW* beam search and graph (Section 3.4): stop rule, threshold, R bound, schedules, heuristic
    ("hnsw_stop_at_the_farthest", "if (kv_less(far.key, far.id, c.key, c.id)) break;", "if (!(c.key < far.key)) break;"),
    ("hnsw_threshold_is_nearest", "const double r2_node = nR == ef ? R[ef - 1].key : INFINITY;",
     "const double r2_node = nR == ef ? R[0].key : INFINITY;"),
    ("hnsw_result_set_unbounded", "if (nR > ef) {", "if (nR > ef + 1) {"),
    ("hnsw_sequential_threshold_stale", "OR_HVISIT(e, nR == ef ? R[ef - 1].key : INFINITY);", "OR_HVISIT(e, r2_node);"),
    ("hnsw_entry_not_exact", "OR_HVISIT(e, INFINITY);", "OR_HVISIT(e, 0.0);"),
    ("hnsw_heuristic_reversed", "if (!(cand[i].key < des)) { keep = 0; break; }",
     "if (!(cand[i].key > des)) { keep = 0; break; }"),
    ("hnsw_reverse_edges_dropped", "for (int64_t t = rstart[v]; t < rstart[v + 1]; ++t) {",
     "for (int64_t t = rstart[v]; t < rstart[v]; ++t) {"),
    ("hnsw_fp32_test_unsquared", "float bound = coef[j] * r2;", "float bound = coef[j] * sqrtf(r2);"),
    ("probe_descending", "for (int j = 0; j < nprobe; ++j) {\n                probe[q * nprobe + j] = (int32_t)buf[j].id;",
     "for (int j = 0; j < nprobe; ++j) {\n                probe[q * nprobe + j] = (int32_t)buf[nc - 1 - j].id;"),
]


def _first_failure(o):
    for pin in pins.ALL:
        try:
            pin(o)
        except Exception as e:  # noqa: BLE001 - any failure counts as caught
            return pin.__name__, type(e).__name__
    return None


@pytest.mark.parametrize("name,old,new", PLANTS, ids=[p[0] for p in PLANTS])
def test_plant_is_caught(name, old, new):
    src = open(oracle.SRC).read()
    olds, news = (old, new) if isinstance(old, list) else ([old], [new])
    for a, b in zip(olds, news):
        assert src.count(a) == 1, f"plant site for {name} not found exactly once"
        src = src.replace(a, b)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "planted.c")
        with open(path, "w") as f:
            f.write(src)
        lib = oracle.build(src=path, out=os.path.join(tmp, "libplanted.so"))
        caught = _first_failure(oracle.Oracle(lib))
    assert caught is not None, f"planted mistake {name} passed every pin"
