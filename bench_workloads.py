"""Secondary measurement lines of bench.py (one JSON line each), same timing rules as the main
line: W >= 3 untimed warm-up steps, CUDA events on the launching stream bracketed by
synchronisations, inputs larger than L2 or resident and stated.

  w1: n=256 SOV, FP64 (Sigma -> Cholesky -> sweep), 10,000 points x 20 shifts.
  w3: confidence region on a posterior field (n=4,096, 256 prefix problems, 10,000 paths):
      one prefix-recording sweep (mvn_excursion) and one batched persistent launch of the 256
      independent problems (mvn_sov_batched), against a loop of single-problem FP64 launches
      (timed on a sample of the problems and scaled by their sample-dims).
  w4: adjoint, n=4,096 Matern 3/2: d log P / d (b, sigma2, range) through the autograd chain.
  w5: tile low rank, n=65,536 exponential (Morton grid), tile 1024, acc 1e-5, max rank 256:
      compression + TLR Cholesky + SOV, against the dense MVN_MIXED factorisation + SOV.
"""
from __future__ import annotations

import json
import time

import numpy as np
import torch

from paper_2405_14892_gb300 import inputs, mvn


def _timed(fn, steps, warmup, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    st, info = mvn.context().sync()
    if st != 0:
        raise RuntimeError(f"device error {st} info {info}")
    return e0.elapsed_time(e1) / steps


def _line(args, workload, metric, value, unit, ms, extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "data": "synthetic", "config": {"workload": workload}}
    d.update(extra)
    print(json.dumps(d), flush=True)


def run(args):
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = mvn.context(0)
    steps, warm = max(1, args.steps), max(3, args.warmup)
    t = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)

    if args.workload == "w1":
        w = inputs.WORKLOADS["W1"]
        c = inputs.grid_coords(w["g"])
        n = c.shape[0]
        a, b = inputs.limits_for(w, n)
        cd, ad, bd = t(c), t(a), t(b)
        S = mvn.colmajor_empty(n, n, dev)
        out3 = torch.empty(3, dtype=torch.float64, device=dev)

        def step():
            mvn.mvn_matern(cd, w["sigma2"], w["range"], w["nu"], w["nugget"], out=S)
            mvn.mvn_cholesky(S, check=False)
            mvn.mvn_sov(ad, bd, S, w["Ns"], w["M"], w["seed"], out3=out3)
        l0 = ctx.launches()
        ms = _timed(step, steps, warm, stream)
        paths = w["Ns"] * w["M"]
        _line(args, w["name"], "SOV sample-dims/s, n=256, FP64", n * paths / (ms * 1e-3),
              "sample-dims/s", ms, {"dtype": "f64", "logP": float(out3[0]),
                                    "gpu_launches": (ctx.launches() - l0) // (steps + warm) * steps})
        return

    if args.workload == "w3":
        w = inputs.WORKLOADS["W3"]
        c = inputs.grid_coords(w["g"])
        n = c.shape[0]
        Sp = mvn.mvn_matern(t(c), w["sigma2"], w["range"], w["nu"], w["nugget"])
        torch.cuda.synchronize()
        Sh = torch.tril(Sp).cpu().numpy()
        Sh = Sh + np.tril(Sh, -1).T
        # synthetic observations of the prior field, then the posterior (Eqs. 7-8) on the GPU
        obs, y, _ = inputs.observations(Sh, w["n_obs"], w["noise_sd"], w["field_seed"])
        od = torch.as_tensor(obs, dtype=torch.int32, device=dev)
        yd = t(y)
        Spost_d = mvn.colmajor_empty(n, n, dev)
        mvn.mvn_posterior(None, Sp, od, yd, w["noise_sd"] ** 2, out_Sigma=Spost_d,
                          prec="mixed")  # warm-up
        res = {}

        def post():
            res["post"] = mvn.mvn_posterior(None, Sp, od, yd, w["noise_sd"] ** 2,
                                            out_Sigma=Spost_d, check=False, prec="mixed")
        ms_post = _timed(post, 1, 1, stream)
        mu = res["post"][0].cpu().numpy()
        Spost = np.tril(Spost_d.cpu().numpy())
        Spost = Spost + np.tril(Spost, -1).T
        dims = inputs.prefix_problem_dims(w["nprob"], w["dims_lo"], w["dims_hi"], w["dims_seed"])
        mud, Sd = t(mu), mvn.to_colmajor(t(Spost))
        tuned = mvn.mvn_autotune(n, w["Ns"] * w["M"], "mixed")

        def exc():
            res["r"] = mvn.mvn_excursion(mud, Sd, w["u"], w["level"], w["Ns"], w["M"], w["seed"],
                                         prefix_dims=dims, prec="mixed")
        ms_exc = _timed(exc, steps, warm, stream)
        r = res["r"]
        # the same pipeline captured once as a CUDA graph: one launch per confidence region
        G = mvn.mvn_excursion_graph(mud, Sd, w["u"], w["level"], w["Ns"], w["M"], w["seed"],
                                    prefix_dims=dims, prec="mixed")
        l0 = ctx.launches()
        ms_graph = _timed(G.launch, steps, warm, stream)
        graph_launches = (ctx.launches() - l0) // (steps + warm) * steps
        if G.sync() != 0:
            raise RuntimeError("graph replay raised a device error")
        same = all(torch.equal(G.result[k], r[k]) for k in ("order", "F", "region"))
        G.close()
        order = r["order"].cpu().numpy()
        Lp = mvn.to_colmajor(t(Spost[np.ix_(order, order)]))
        mvn.mvn_cholesky(Lp)
        a_perm = t(w["u"] - mu[order])
        b_inf = t(np.full(n, np.inf))

        def batched():
            res["b"] = mvn.mvn_sov_batched(dims, [0] * len(dims), a_perm, b_inf, Lp, w["Ns"],
                                           w["M"], w["seed"], prec="mixed")
        ms_bat = _timed(batched, steps, warm, stream)
        # loop of single-problem FP64 launches, on a sample of 8 problems, scaled by sample-dims
        sample = list(range(0, len(dims), len(dims) // 8))[:8]

        def loop():
            for p in sample:
                k = int(dims[p])
                mvn.mvn_sov(a_perm[:k].contiguous(), b_inf[:k].contiguous(), Lp, w["Ns"], w["M"],
                            w["seed"], prec="fp64")
        ms_loop_sample = _timed(loop, 1, 1, stream)
        sd_sample = sum(int(dims[p]) ** 2 for p in sample)
        sd_all = sum(int(k) ** 2 for k in dims)
        ms_loop = ms_loop_sample * sd_all / sd_sample
        _line(args, w["name"],
              "confidence-region MVN probs/s (256 prefix problems, one sweep, one graph launch)",
              len(dims) / (ms_graph * 1e-3), "probs/s", ms_graph,
              {"dtype": "f64+f32+fp16x2+bf16 digits", "eager_ms": ms_exc,
               "eager_probs_per_sec": len(dims) / (ms_exc * 1e-3),
               "graph_equals_eager": bool(same), "gpu_launches": graph_launches,
               "launch_shapes_autotuned": tuned,
               "kernels_per_graph": G.kernels, "batched_independent_ms": ms_bat,
               "posterior_ms": ms_post,
               "batched_probs_per_sec": len(dims) / (ms_bat * 1e-3),
               "loop_fp64_single_ms_estimated": ms_loop,
               "loop_sample": f"{len(sample)} of {len(dims)} problems timed, scaled by sum k^2",
               "region_size": int(r["region"].sum()), "F_first_last": [float(r["F"][0]),
                                                                       float(r["F"][-1])]})
        return

    if args.workload == "w4":
        from paper_2405_14892_gb300.autograd import mvn_log_prob
        w = inputs.WORKLOADS["W4"]
        c = t(inputs.grid_coords(w["g"]))
        n = c.shape[0]
        _, b = inputs.limits_for(w, n)
        res, ms, kms = {}, {}, {}
        names = ("k_sov_grad_fwd_f64", "k_sov_grad_fwd_f32", "k_sov_rev_f64", "k_sov_rev_f32",
                 "k_grad_L_f64", "k_grad_L_f32", "k_oz_update", "k_oz_potrf", "k_oz_trsm",
                 "k_syrk", "k_gemm64", "k_cgrad_panel", "k_cgrad_diag")
        for prec in ("mixed", "fp64"):
            bt = t(b).requires_grad_(True)
            s2 = torch.tensor(w["sigma2"], dtype=torch.float64, device=dev, requires_grad=True)
            rg = torch.tensor(w["range"], dtype=torch.float64, device=dev, requires_grad=True)

            def step():
                bt.grad = None
                s2.grad = None
                rg.grad = None
                lp = mvn_log_prob(bt, s2, rg, c, nu=w["nu"], nugget=w["nugget"],
                                  n_points=w["Ns"], n_shifts=w["M"], seed=w["seed"], prec=prec)
                lp.backward()
                res[prec] = lp.detach()
            ms[prec] = _timed(step, steps, warm, stream)
            res[prec] = (float(res[prec]), bt.grad.cpu().numpy(), float(s2.grad), float(rg.grad))
            # per-kernel device time of one more step, from the library's own events
            ctx.timing(True)
            keep = res[prec]
            step()
            res[prec] = keep
            torch.cuda.synchronize()
            kms[prec] = {k: round(v[0], 3) for k in names
                         for v in [ctx.kernel_time(k)] if v[1]}
            ctx.timing(False)
        l64, gb64, s64, r64 = res["fp64"]
        lmx, gbmx, smx, rmx = res["mixed"]
        _line(args, w["name"], "gradients/s of log P w.r.t. (b, sigma2, range), n=4096",
              1e3 / ms["mixed"], "gradients/s", ms["mixed"],
              {"dtype": "f64+f32 (mixed) vs f64", "fp64_ms": ms["fp64"],
               "fp64_gradients_per_sec": 1e3 / ms["fp64"],
               "mixed_over_fp64_speedup": ms["fp64"] / ms["mixed"],
               "logP": {"mixed": lmx, "fp64": l64},
               "mixed_vs_fp64": {"dlogP": abs(lmx - l64),
                                 "db_rel": float(np.abs(gbmx - gb64).max() /
                                                 max(1.0, np.abs(gb64).max())),
                                 "dsigma2_rel": abs(smx - s64) / max(1.0, abs(s64)),
                                 "drange_rel": abs(rmx - r64) / max(1.0, abs(r64))},
               "dsigma2": smx, "drange": rmx, "kernel_ms_one_step": kms})
        return

    if args.workload == "w6":
        # confidence-region detection at the paper's synthetic scale (Sec. V-B): 40,000 sites,
        # 6,250 noisy observations -> posterior (Eqs. 7-8, MVN_MIXED) -> Alg. 1 over every prefix
        w = inputs.WORKLOADS["W6"]
        c = inputs.grid_coords(w["g"])
        n = c.shape[0]
        Sp = mvn.mvn_matern(t(c), w["sigma2"], w["range"], w["nu"], w["nugget"])
        torch.cuda.synchronize()

        def block(idx):
            ii = torch.as_tensor(idx, dtype=torch.int64, device=dev)
            Lo = torch.tril(Sp[ii][:, ii])
            return (Lo + Lo.t() - torch.diag(torch.diag(Lo))).cpu().numpy()
        obs, y, _ = inputs.observations_at_sites(n, w["n_obs"], w["noise_sd"], w["field_seed"],
                                                 block)
        od = torch.as_tensor(obs, dtype=torch.int32, device=dev)
        yd = t(y)
        Spost = mvn.colmajor_empty(n, n, dev)
        res = {}

        def post():
            res["post"] = mvn.mvn_posterior(None, Sp, od, yd, w["noise_sd"] ** 2,
                                            out_Sigma=Spost, check=False, prec="mixed")
        ms_post = _timed(post, 1, 1, stream)
        mu = res["post"][0]

        def exc():
            res["r"] = mvn.mvn_excursion(mu, Spost, w["u"], w["level"], w["Ns"], w["M"], w["seed"],
                                         prec="mixed")
        ms_exc = _timed(exc, 1, 1, stream)
        r = res["r"]
        F = r["F"].cpu().numpy()
        region = int(r["region"].sum().item())
        total = ms_post + ms_exc
        _line(args, w["name"], "confidence regions/s, n=40,000 sites, 6,250 observations",
              1e3 / total, "regions/s", total,
              {"dtype": "posterior: exact-digit tensor-core Schur complement + double-float panel; "
                        "excursion: f64+f32+fp16x2+bf16 digits",
               "posterior_ms": ms_post, "excursion_ms": ms_exc, "region_sites": region,
               "F_first": [float(x) for x in F[:3]], "F_last": float(F[-1]),
               "prefixes": int(F.size), "paths": w["Ns"] * w["M"],
               "note": "one warm-up and one timed call of each stage"})
        return

    if args.workload == "w5":
        w = inputs.WORKLOADS["W5"]
        c = inputs.grid_coords(w["g"], order="morton")
        n = c.shape[0]
        a, b = inputs.limits_for(w, n)
        cd, ad, bd = t(c), t(a), t(b)
        S = mvn.colmajor_empty(n, n, dev)
        Lt = mvn.colmajor_empty(n, n, dev)
        out_t = torch.empty(3, dtype=torch.float64, device=dev)
        out_d = torch.empty(3, dtype=torch.float64, device=dev)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        out_x = torch.empty(3, dtype=torch.float64, device=dev)
        mvn.mvn_matern(cd, w["sigma2"], w["range"], w["nu"], w["nugget"], out=S)
        torch.cuda.synchronize()
        ctx.timing(True)
        e[0].record(stream)
        T = mvn.mvn_tlr_compress(S, w["tile"], w["acc"], w["max_rank"])
        e[1].record(stream)
        mvn.mvn_tlr_cholesky(T)
        e[2].record(stream)
        # the sweep on the compressed factor (low-rank limit updates, FP32 shifts)
        mvn.mvn_sov_tlr(T, ad, bd, w["Ns"], w["M"], w["seed"], prec="mixed", out3=out_t)
        e[3].record(stream)
        # for comparison: the factor expanded to dense and the tensor-core sweep
        Lt.zero_()
        mvn.mvn_tlr_to_dense(T, out=Lt)
        mvn.mvn_sov(ad, bd, Lt, w["Ns"], w["M"], w["seed"], prec="mixed", out3=out_x)
        e[4].record(stream)
        mvn.mvn_cholesky(S, prec="mixed", check=False)
        e[5].record(stream)
        mvn.mvn_sov(ad, bd, S, w["Ns"], w["M"], w["seed"], prec="mixed", out3=out_d)
        e[6].record(stream)
        torch.cuda.synchronize()
        mvn.sync()
        kms = {k: round(v[0], 2) for k in ("k_bgemm", "k_chol_inv", "k_jacobi1", "k_trsm_block",
                                           "k_syrk", "k_oz_update", "k_oz_potrf", "k_oz_trsm",
                                           "k_sov_tc", "k_sov_tlr_f32")
               for v in [ctx.kernel_time(k)] if v[1]}
        ctx.timing(False)
        ms = [e[i].elapsed_time(e[i + 1]) for i in range(6)]
        ranks = T.ranks()
        tlr_ms = ms[0] + ms[1] + ms[2]
        dense_ms = ms[4] + ms[5]
        _line(args, w["name"], "TLR vs dense time-to-P-hat, n=65,536", 1e3 / tlr_ms, "probs/s",
              tlr_ms, {"dtype": "f64 (TLR factor) + f32 low-rank sweep / f64+f32+fp16x2+bf16 "
                                "digits (dense)",
                       "tlr_compress_ms": ms[0], "tlr_cholesky_ms": ms[1],
                       "tlr_sov_lowrank_ms": ms[2], "tlr_sov_expanded_ms": ms[3],
                       "dense_cholesky_ms": ms[4], "dense_sov_ms": ms[5],
                       "tlr_over_dense_speedup": dense_ms / tlr_ms,
                       "sov_lowrank_over_dense": ms[5] / ms[2],
                       "logP_tlr": float(out_t[0]), "logP_tlr_expanded": float(out_x[0]),
                       "logP_dense": float(out_d[0]),
                       "ranks": {"min": int(ranks.min()), "median": float(np.median(ranks)),
                                 "max": int(ranks.max()), "capped": int(T.capped)},
                       "kernel_ms": kms,
                       "note": "single timed pass (no warm-up repeats: minutes per pass)"})
        return
