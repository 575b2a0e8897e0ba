"""Performance model of Sec. 5 (host-side arithmetic, no device code).

Eq. (A_gm):  A_gm(D) = N (L_gm + S_gm) = 2 N D_uncache + 2 D_cache    [cells]
Eq. (time_gm): T_gm = A_gm * S(type) / B_gm
Eq. (A_sm):  A_sm = 2 (N - 1) D_cache^sm                                [cells]
Eq. (time_sm): T_sm = (A_sm + A_sm(KERNEL)) * S(type) / B_sm
Eq. (maxlat): T_PERKS = max(T_gm, T_sm)
Eq. (maxpeak): P = D N / T_PERKS

The worked example of Sec. 5.2 (single-precision 2d5pt, 3072^2 cells, 1000
steps, A100 at 1555 GB/s) adds the halo traffic of the cached tiles as a
separate time term and sums it with T_gm; its printed numbers (9900.70 us,
871.22 us, 876.09 GCells/s) are reproduced only by that sum, so
``worked_example_time`` follows it.  Sec. 5.3: the efficiency function is 1
when the software concurrency covers the hardware concurrency, which Little's
law gives as throughput x latency.

``stencil_algorithmic_bytes`` is the roofline numerator used by the bench:
the bytes the persistent method must move per run (uncached cells read and
written every step, cached cells loaded and stored once, halo cells written
and read every step).
"""
from __future__ import annotations


def global_cells_accessed(d_cells: float, d_cache_cells: float, n_steps: int) -> float:
    """A_gm in cells: 2 N D_uncache + 2 D_cache."""
    d_uncache = d_cells - d_cache_cells
    return 2.0 * n_steps * d_uncache + 2.0 * d_cache_cells


def t_gm(d_cells: float, d_cache_cells: float, n_steps: int, elem_bytes: int,
         bw_bytes_per_s: float) -> float:
    return global_cells_accessed(d_cells, d_cache_cells, n_steps) * elem_bytes / bw_bytes_per_s


def sm_cells_accessed(d_cache_sm_cells: float, n_steps: int) -> float:
    """A_sm in cells: 2 (N-1) D_cache^sm."""
    return 2.0 * (n_steps - 1) * d_cache_sm_cells


def t_sm(d_cache_sm_cells: float, n_steps: int, kernel_sm_cells: float, elem_bytes: int,
         bw_sm_bytes_per_s: float) -> float:
    return ((sm_cells_accessed(d_cache_sm_cells, n_steps) + kernel_sm_cells) * elem_bytes
            / bw_sm_bytes_per_s)


def t_perks(tgm: float, tsm: float) -> float:
    return max(tgm, tsm)


def projected_peak_cells_per_s(d_cells: float, n_steps: int, t_seconds: float) -> float:
    return d_cells * n_steps / t_seconds


def halo_time(halo_cells: float, elem_bytes: int, bw_bytes_per_s: float) -> float:
    return halo_cells * elem_bytes / bw_bytes_per_s


def worked_example_time(d_cells, d_cache_cells, n_steps, halo_cells, elem_bytes, bw):
    """(T_gm, T_halo, total) as the Sec. 5.2 example combines them."""
    a = t_gm(d_cells, d_cache_cells, n_steps, elem_bytes, bw)
    h = halo_time(halo_cells, elem_bytes, bw)
    return a, h, a + h


def hardware_concurrency(throughput_per_cycle: float, latency_cycles: float) -> float:
    """Little's law: C_hw = THR * L."""
    return throughput_per_cycle * latency_cycles


def sm_software_concurrency(per_block: float, blocks_per_sm: int) -> float:
    """C_sw^SM = C_sw^TB * TB/SM."""
    return per_block * blocks_per_sm


def efficiency(c_sw: float, c_hw: float) -> float:
    """E = 100 % when the exposed concurrency covers the hardware's; below
    that the paper leaves E unmodelled, and this returns the ratio."""
    return 1.0 if c_sw >= c_hw else c_sw / c_hw


def stencil_algorithmic_bytes(d_cells: float, d_cache_cells: float, n_steps: int,
                              halo_cells_per_step: float, elem_bytes: int) -> float:
    """S * (2 N D_uncache + 2 D_cache) + S * N * H, H = halo cells written+read per step."""
    return elem_bytes * (global_cells_accessed(d_cells, d_cache_cells, n_steps)
                         + n_steps * halo_cells_per_step)
