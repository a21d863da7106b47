"""B300-native Kadir-Brady 3D saliency: spherical-window histograms and
entropies for the dense sweep and the two seed-climbing schemes.

Import `paper_1310_6736_b300.ks` for the C-ABI binding; importing the
package itself loads nothing native.
"""
