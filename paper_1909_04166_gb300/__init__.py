"""GB300 (sm_103a) implementation of the per-time-step update of the coupled cascaded
central-moment lattice Boltzmann schemes of Hajabdollahi, Premnath & Welch (arXiv:1909.04166).
"""
