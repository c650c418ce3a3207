"""CPU oracle of the exact ray-Gaussian renderer. Test infrastructure only."""
