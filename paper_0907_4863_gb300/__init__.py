"""GB300-native SAAMG-PCG: CG on the finite-difference Poisson system of an irregular
3-D pipe domain, preconditioned by a smoothed-aggregation AMG V-cycle."""
