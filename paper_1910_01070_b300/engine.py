"""Convenience layer over the C ABI: one context with its resident tables and
setups, built from the seeded workload descriptions.  Argument marshalling
only; all arithmetic of the forward model runs in libhr2.so."""
from __future__ import annotations

from typing import Dict, List, Optional

import numpy as np

from . import hr2
from . import workloads as W

STORAGE = {"fp16": hr2.HR2_STORE_FP16_OFFSET, "fp64": hr2.HR2_STORE_FP64}


class Engine:
    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.ctx = hr2.hr2_ctx_create(device, mem_budget_bytes)
        self.device = device
        self.tables = []
        self.setups = []

    # ------------------------------------------------------------ objects
    def add_tables(self, spec: W.TableSpec, storage: str = "fp16", arrays: Optional[Dict] = None):
        """Create device tables.  With ``arrays`` (log10_sigma etc. as float64) they are uploaded at once;
        otherwise each species is generated and uploaded in turn (bounded host memory)."""
        st = STORAGE[storage]
        if arrays is not None:
            h = hr2.create_opacity_tables(self.ctx, arrays["T_grid"], arrays["log10p_grid"], arrays["nu0"],
                                          arrays["dnu"], arrays["log10_sigma"].shape[-1], arrays["species_mass"],
                                          arrays["log10_sigma"], arrays.get("log10_cia_h2h2"),
                                          arrays.get("log10_cia_h2he"), st)
        else:
            h2h2, h2he = W.cia_tables(spec)
            h = hr2.create_opacity_tables(self.ctx, spec.T_grid, spec.log10p_grid, spec.nu0, spec.dnu, spec.n_nu,
                                          spec.masses, None, h2h2, h2he, st)
            for s in range(spec.n_species):
                hr2.hr2_tables_upload_species(self.ctx, h, s, W.species_table(spec, s))
        self.tables.append(h)
        return h

    def add_setup(self, tables, s: W.SetupSpec, obs_flux=None, obs_sigma=None, level_cache=True):
        """A setup on the engine's tables.  level_cache: True (the level-gridded operand, built
        once), False (the FP16 tables read directly), "auto" (the operand where it fits, else
        streamed) or "stream" (the operand built per call and group of tiles into a ring)."""
        h = hr2.hr2_setup_create(self.ctx, tables, s.nu_first, s.n_nu, s.n_layers, s.species, s.n_mu,
                                 s.fe_elements, s.fe_order, s.resolving_power, s.bin_edges, s.p_top, s.p_bot,
                                 s.r_he, s.radius_cm, obs_flux, obs_sigma, level_cache, s.interp, s.profile, s.cloud, s.sc)
        self.setups.append(h)
        return h

    def set_observation(self, setup, D, sigma):
        hr2.hr2_setup_set_observation(self.ctx, setup, D, sigma)

    def set_launch_config(self, warps_per_cta: int, ctas_per_sm: int, tiles_per_item: int = 1, stages: int = 0,
                          split_max_batch: int = 2):
        hr2.hr2_set_launch_config(self.ctx, warps_per_cta, ctas_per_sm, tiles_per_item, stages, split_max_batch)

    def memory(self):
        return hr2.hr2_ctx_memory(self.ctx)

    def close(self):
        if self.ctx is not None:
            hr2.hr2_ctx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ batches
    def forward(self, setups: List, setup_of_sample, params, out_bins=None, out_highres=None, out_status=None,
                stream=None):
        import torch
        n = params.shape[0]
        if out_bins is None:
            nb = max(hr2.hr2_setup_info(s)[0] for s in setups)
            out_bins = torch.empty((n, nb), dtype=torch.float32, device=params.device)
        hr2.forward_model_batch(self.ctx, setups, setup_of_sample, params, out_bins, out_highres, out_status, stream)
        return out_bins

    def lnl(self, setups: List, setup_of_sample, model_bins, log_eps=None, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(model_bins.shape[0], dtype=torch.float64, device=model_bins.device)
        hr2.log_likelihood_batch(self.ctx, setups, setup_of_sample, model_bins, out, log_eps, stream)
        return out

    def evaluate_host(self, setups: List, setup_of_sample, params, log_eps=None, out_bins=None, stream=None):
        n = params.shape[0]
        out = np.empty(n, dtype=np.float64)
        hr2.hr2_evaluate_host(self.ctx, setups, setup_of_sample, params, out, log_eps, out_bins, stream)
        return out


def build_workload(eng: Engine, wl: W.Workload, storage: Optional[str] = None, arrays: Optional[Dict] = None):
    """Tables and setups of a workload on the engine; returns (tables, [setups])."""
    t = eng.add_tables(wl.table, storage or wl.storage, arrays)
    return t, [eng.add_setup(t, s) for s in wl.setups]
